"""The C-ABI library loads and exports every declared symbol; plan creation
validates its arguments (host logic only, no GPU work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lramm.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lramm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    import paper_2405_16917_gb300 as L
    if not os.path.exists(L.LIB_PATH):
        from paper_2405_16917_gb300 import _build
        _build.build()
    L.load()
    return L


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("lramm_plan_create", "lramm_rsvd", "lramm_matmul", "lramm_chain", "lramm_workspace_size",
              "lramm_plan_destroy", "lramm_status_read", "lramm_quantize", "lramm_qgemm",
              "lramm_gaussian", "lramm_philox_words"):
        assert s in syms


def test_library_exports_every_declared_symbol(L):
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(L):
    assert set(declared_symbols()) <= set(L._SIGS)


def _plan(L, **kw):
    args = dict(m=512, n=512, k=512, r=64, p=10, q=1)
    args.update(kw)
    return L.Plan(**args)


def test_plan_create_and_workspace(L):
    p = _plan(L)
    assert p.ws_bytes > 0 and p.ws_bytes % 256 == 0
    big = _plan(L, m=4096, n=4096, k=4096, r=256, p=16, q=2)
    assert big.ws_bytes > p.ws_bytes
    p.close()
    big.close()


@pytest.mark.parametrize("kw", [dict(m=0), dict(r=0), dict(p=-1), dict(q=17), dict(r=500, p=20),
                                dict(lda=100), dict(prec=(9, 1, 1)), dict(scale=5), dict(sketch=7),
                                dict(a_type=3)])
def test_plan_rejects_invalid(L, kw):
    with pytest.raises(L.LrammError) as e:
        _plan(L, **kw)
    assert e.value.code == 1


def test_plan_unsupported_sketch_width(L):
    with pytest.raises(L.LrammError) as e:
        _plan(L, m=4096, n=4096, k=4096, r=500, p=30)
    assert e.value.code == 2


def test_calls_reject_bad_arguments_without_gpu_work(L):
    lib = L.load()
    p = _plan(L)
    nul = ctypes.c_void_p(0)
    assert lib.lramm_matmul(p.handle, nul, nul, nul, nul, nul, 0, nul) == 1
    assert lib.lramm_rsvd(p.handle, 2, nul, nul, nul, nul, nul, 0, nul) == 1
    fake = ctypes.c_void_p(256)
    assert lib.lramm_matmul(p.handle, fake, fake, nul, fake, fake, 16, nul) == 3     # workspace too small
    assert lib.lramm_matmul(p.handle, fake, fake, nul, fake, ctypes.c_void_p(300), p.ws_bytes, nul) == 3
    assert lib.lramm_qgemm(fake, fake, 4, 4, 17, 17, 17, 1, 1, fake, fake, 1.0, 0.0, nul, 0, fake, 4, 0,
                           nul) == 1                                                   # K % 16
    assert lib.lramm_qgemm_tc(1, fake, fake, 4, 4, 17, 17, 17, 1, fake, fake, 1.0, 0.0, nul, 0, fake, 4, fake, 4096,
                              nul) == 1                                                # K % 16
    assert lib.lramm_qgemm_tc(1, fake, fake, 4, 4, 16, 16, 16, 1, fake, fake, 1.0, 0.0, nul, 0, fake, 4, nul, 0,
                              nul) == 3                                                # no workspace
    assert lib.lramm_qgemm_tc(0, fake, fake, 4, 4, 16, 16, 16, 1, fake, fake, 1.0, 0.0, nul, 0, fake, 4, fake, 4096,
                              nul) == 1                                                # F32 is not a code
    assert lib.lramm_qgemm_tc_ws_bytes(1, 256, 256, 4096) > lib.lramm_qgemm_tc_ws_bytes(1, 256, 256, 256)
    assert lib.lramm_tgemm_tc(4, 4, 8, 1.0, fake, 4, fake, 8, 0.0, fake, 4, fake, 4096, nul) == 1   # lda < K
    assert lib.lramm_tgemm_tc(4, 4, 8, 1.0, fake, 8, fake, 8, 0.0, fake, 4, nul, 0, nul) == 3       # no workspace
    assert lib.lramm_quantize(fake, 4, 8, 8, 0, 1, fake, 8, fake, nul, nul) == 1      # F32 is not a code
    assert lib.lramm_philox_words(1, 0, 4, ctypes.c_void_p(4), nul) == 1               # misaligned
    assert lib.lramm_status_str(5).decode().startswith("non-positive")


def test_plan_validates_lead_tail_fields(L):
    ok = _plan(L, prec=(1, 1, 4), lead=16, lead_prec=1, lead_split=2)
    ok.close()
    for bad in (dict(lead=65), dict(lead=-1), dict(lead=8, lead_prec=0), dict(lead=8, lead_prec=4),
                dict(lead=8, lead_split=3)):
        with pytest.raises(L.LrammError) as e:
            _plan(L, **bad)
        assert e.value.code == 1, bad
    with pytest.raises(L.LrammError) as e:
        _plan(L, prec=(1, 1, 5))
    assert e.value.code == 1


def test_plan_l_limits(L):
    # l = 576 is the orthonormalisation's limit (two-level Cholesky), 580 is past it
    p = _plan(L, m=2048, n=2048, k=2048, r=560, p=16)
    p.close()
    with pytest.raises(L.LrammError) as e:
        _plan(L, m=2048, n=2048, k=2048, r=564, p=16)
    assert e.value.code == 2
    # l = 342 (not a multiple of 4, past the column-panel Cholesky's shared memory) is refused
    with pytest.raises(L.LrammError) as e:
        _plan(L, m=2048, n=2048, k=2048, r=326, p=16)
    assert e.value.code == 2


def test_dq_and_mx_argument_checks(L):
    lib = L.load()
    fake, nul = ctypes.c_void_p(256), ctypes.c_void_p(0)
    assert lib.lramm_dq_matmul(0, 0, 4, 4, 4, 1.0, fake, 4, fake, 4, 0.0, nul, 0, fake, 4, fake, 1 << 20, nul) == 1
    assert lib.lramm_dq_matmul(1, 2, 4, 4, 4, 1.0, fake, 4, fake, 4, 0.0, nul, 0, fake, 4, fake, 1 << 20, nul) == 1
    assert lib.lramm_dq_matmul(1, 0, 4, 4, 4, 1.0, fake, 4, fake, 4, 0.0, nul, 0, fake, 4, nul, 0, nul) == 3
    assert lib.lramm_dq_ws_bytes(1, 4096, 4096, 4096) > lib.lramm_dq_ws_bytes(1, 64, 64, 64)
    assert lib.lramm_quantize_mx(fake, 4, 40, 40, fake, 40, fake, nul) == 1       # ldcodes not a multiple of 32
    assert lib.lramm_qgemm_mx(fake, fake, fake, fake, 4, 4, 48, 48, 48, 1.0, 0.0, nul, 0, fake, 4, nul) == 1
    assert lib.lramm_launch_count() >= 0


def test_qsvd_argument_checks(L):
    lib = L.load()
    p = _plan(L)
    fake, nul, bad = ctypes.c_void_p(256), ctypes.c_void_p(0), ctypes.c_void_p(264)
    I8, I4, E4, MX = L.P_INT8, L.P_INT4, L.P_E4M3, L.P_MXFP4

    def call(which=0, pu=I8, pv=I8, Uc=fake, ldq=64, Xr=fake, ws=fake, wsb=None):
        return lib.lramm_qsvd(p.handle, which, fake, pu, pv, Uc, fake, fake, fake, ldq, nul, nul, Xr,
                              4096, ws, p.ws_bytes if wsb is None else wsb, nul)
    assert call(which=2) == 1
    assert call(pu=MX) == 2                       # MXFP4 factors: not offered
    assert call(pv=0) == 1                        # F32 is not a code format
    assert call(ldq=80) == 1                      # ldq a multiple of 32
    assert call(ldq=32) == 1                      # ldq >= r
    assert call(Uc=bad) == 1                      # codes 16-byte aligned
    assert call(pu=I8, pv=E4) == 2                # no common code product for INT8 / E4M3 ...
    assert call(pu=I8, pv=E4, Xr=nul, wsb=16) == 3   # ... but the codes alone are fine
    assert call(wsb=16) == 3                      # workspace too small
    assert lib.lramm_qsvd_ws_bytes(p.handle, 0, I8, I8) >= p.ws_bytes
    assert lib.lramm_qsvd_ws_bytes(p.handle, 0, I8, I4) > lib.lramm_qsvd_ws_bytes(p.handle, 0, I8, I8)
    assert lib.lramm_qsvd_ws_bytes(p.handle, 1, MX, I8) == 0
    assert lib.lramm_kernel_kind_name(16).decode() == "reconstruct"
    assert lib.lramm_kernel_kind_name(17).decode() == "unknown"
