"""The allocation-free quantiser (lramm_quantize_noalloc) against lramm_quantize.

Some callers cannot allocate device memory themselves (their framework owns
all GPU memory through its own pool, or their host gives plug-ins no
allocator); lramm_quantize_noalloc serves them by keeping its per-tensor
a_max accumulator in an array inside the library.  Its codes and scales must
be exactly those of lramm_quantize (the quantiser tests' bar: bit-exact),
on two calls in a row -- the second with a smaller a_max than the first, so
an accumulator that was not cleared between calls would show.

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process (the
first call on the device looks up the array's address).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_noalloc_quantize_matches_workspace_quantize_twice(L, prec):
    rng = np.random.default_rng(40 + prec)
    first = (rng.standard_normal((150, 97)) * 50.0).astype(np.float32)
    second = (rng.standard_normal((61, 33)) * 0.01).astype(np.float32)
    for X in (first, second):
        Xd = torch.from_numpy(X).cuda()
        ld = X.shape[1] + (-X.shape[1]) % 16
        codes = torch.empty((X.shape[0], ld), dtype=L.code_dtype(prec), device="cuda")
        scales = torch.empty((1,), dtype=torch.float32, device="cuda")
        c_na, s_na = L.quantize_noalloc(Xd, prec, per_row=False, ldcodes=ld, codes=codes, scales=scales)
        c_ws, s_ws = L.quantize(Xd, prec, per_row=False, ldcodes=ld)
        torch.cuda.synchronize()
        assert torch.equal(c_na.float(), c_ws.float())
        assert torch.equal(s_na, s_ws)
        assert s_na.item() == np.float32(np.abs(X).max()) / np.float32({1: 127, 2: 7, 3: 448}[prec])


def test_noalloc_scratch_is_modest(L):
    assert L.load().lramm_noalloc_scratch_bytes() == 256
