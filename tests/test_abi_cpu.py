"""CPU checks of the C ABI library: it builds for sm_103a, loads, and exports every entry point that
include/cakf.h declares; host-side argument validation.  No compute call runs here (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_08971_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            src = open(os.path.join(ROOT, "include", hdr)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|const char\*)\s+(cakf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cakf_filter", "cakf_smooth", "cakf_nll", "cakf_nll_backward"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_struct_matches_header_field_order():
    from paper_2405_08971_gb300 import binding
    src = open(os.path.join(ROOT, "include", "cakf.h")).read()
    body = src[src.index("typedef struct {"):src.index("} cakf_problem;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)\s*;", body)
    assert fields == [f for f, _ in binding.cakf_problem._fields_]


def test_argument_validation_on_host(lib):
    """Invalid arguments are rejected before any device work (ERR_ARG, message set)."""
    from paper_2405_08971_gb300 import binding as b
    coords = np.zeros((4, 2))
    p, keep = b.make_problem(coords, 1, 0.0, 0.0, 0.0, 0.0, T=1, dt=0.1, obs_ptr=[0, 2], obs_idx=[0, 7],
                             y=[1.0, 2.0], budget_i=2, rank_r=0)
    ctx = b.Context()
    with pytest.raises(b.CakfError) as ei:
        b.cakf_filter((p, keep), ctx)
    assert ei.value.code == b.ERR_ARG and "range" in str(ei.value)
    p, keep = b.make_problem(coords, 1, 0.0, 0.0, 0.0, 0.0, T=1, dt=0.1, obs_ptr=[0, 2], obs_idx=[1, 1],
                             y=[1.0, 2.0], budget_i=2, rank_r=0)
    with pytest.raises(b.CakfError) as ei:
        b.cakf_filter((p, keep), ctx)
    assert ei.value.code == b.ERR_ARG and "duplicate" in str(ei.value)
    p, keep = b.make_problem(coords, 5, 0.0, 0.0, 0.0, 0.0, T=1, dt=0.1, obs_ptr=[0, 1], obs_idx=[1],
                             y=[1.0], budget_i=2, rank_r=0)
    with pytest.raises(b.CakfError) as ei:
        b.cakf_filter((p, keep), ctx)
    assert ei.value.code == b.ERR_ARG
    with pytest.raises(b.CakfError) as ei:
        b.cakf_smooth(ctx)
    assert ei.value.code == b.ERR_STATE   # no filter has created a context yet
    for call in (b.cakf_nll, b.cakf_nll_backward):
        with pytest.raises(b.CakfError) as ei:
            call(ctx)
        assert ei.value.code == b.ERR_STATE


def test_gram_wrappers_check_shapes_before_any_launch():
    """The Gram x matrix wrappers reject operands whose shapes disagree (a shorter or narrower Xc
    would make the library read past it) and operands off the current CUDA device, with ValueError,
    before the library is called."""
    torch = pytest.importorskip("torch")
    from paper_2405_08971_gb300 import binding as b
    f64, f32 = torch.float64, torch.float32
    Xr = torch.zeros((10, 2), dtype=f64)
    good = dict(Xc=torch.zeros((7, 2), dtype=f64), B=torch.zeros((3, 7), dtype=f32), out=torch.zeros((3, 10), dtype=f32))
    bad = [dict(good, Xc=torch.zeros((6, 2), dtype=f64)),       # B has 7 rows per column
           dict(good, Xc=torch.zeros((7, 1), dtype=f64)),       # narrower than Xr
           dict(good, Xc=torch.zeros((7, 4), dtype=f64)),       # dim 4
           dict(good, B=torch.zeros((3, 8), dtype=f32)),
           dict(good, out=torch.zeros((3, 9), dtype=f32)),
           dict(good, out=torch.zeros((4, 10), dtype=f32)),
           dict(good, B=torch.zeros((3, 7), dtype=f64))]       # wrong element type for fp32
    for case in bad:
        with pytest.raises(ValueError):
            b.cakf_gram_matmul_noalloc(1, 0.0, 0.0, Xr, case["Xc"], case["B"], case["out"], precision="fp32")
        if case["B"].dtype == f32:   # cakf_gram_matmul converts B to the element type first
            with pytest.raises(ValueError):
                b.cakf_gram_matmul(1, 0.0, 0.0, Xr, case["Xc"], case["B"], out=case["out"], precision="fp32")
    # well-formed host tensors are still refused: the library works on the current CUDA device
    with pytest.raises(ValueError, match="CUDA"):
        b.cakf_gram_matmul_noalloc(1, 0.0, 0.0, Xr, good["Xc"], good["B"], good["out"], precision="fp32")
