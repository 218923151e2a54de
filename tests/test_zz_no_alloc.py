"""nst_gram_noalloc: the Gram statistics for callers that may not allocate device memory.

Its result must equal that of the allocating entry point nst_gram on the same input, call after
call: the library-resident scratch array keeps the previous call's contents, so consecutive
calls with different inputs are checked. Both entries use the same kernels and chunk plan, so
the two results are bitwise equal as well as within the Gram tests' tolerance. Kept in a file of
its own that runs last.
"""
import pytest
import torch

from paper_2212_13459_gb300 import build, native

pytestmark = pytest.mark.gpu

TOL = 1e-6   # the Gram tests' tolerance


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    native.lib()


def _check_pair(V):
    C = V.shape[1]
    ref = torch.empty((C, C), dtype=torch.float64, device="cuda")
    native.gram(V, ref)
    out = torch.full((C, C), 11.0, dtype=torch.float64, device="cuda")
    native.gram_noalloc(V, out)
    torch.cuda.synchronize()
    assert ((out - ref).norm() / ref.norm()).item() <= TOL
    assert torch.equal(out, ref)
    exact = V.double().T @ V.double()
    assert ((out - exact).norm() / exact.norm()).item() <= TOL


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_noalloc_matches_allocating_entry_on_consecutive_calls(dtype):
    g = torch.Generator(device="cuda").manual_seed(21)
    V1 = torch.rand(70001, 512, device="cuda", generator=g).to(dtype)
    V2 = (torch.rand(1000, 64, device="cuda", generator=g) * 3.0).to(dtype)
    V3 = torch.rand(4097, 256, device="cuda", generator=g).to(dtype)
    _check_pair(V1)   # first call: large, fills many scratch blocks
    _check_pair(V2)   # second call: smaller, stale blocks from the first call remain
    _check_pair(V3)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    V = torch.rand(100, 576, device="cuda")
    G = torch.zeros((576, 576), dtype=torch.float64, device="cuda")
    with pytest.raises(native.NSTError) as e:
        native.gram_noalloc(V, G)
    assert e.value.code == native.NST_ERR_SHAPE
    assert "scratch" in str(e.value)
    # a channel count that is not a multiple of 64 is an argument error, as for nst_gram
    V = torch.rand(100, 96, device="cuda")
    G = torch.zeros((96, 96), dtype=torch.float64, device="cuda")
    for fn in (native.gram, native.gram_noalloc):
        with pytest.raises(native.NSTError) as e:
            fn(V, G)
        assert e.value.code == native.NST_ERR_INVALID_ARG
