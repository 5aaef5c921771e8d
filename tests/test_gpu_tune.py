"""Parameter tuning (Sec. 3.5) on the device: the probe error estimate
against the oracle's on the same probes (FP32 products: 1e-4), against the
exact error (16 probes: 25%), and the selection rule applied to the
measured candidates."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


def _operands(n, seed):
    sig = workloads.spectrum("poly1", n)
    A = workloads.lowrank(n, n, sig, seed).astype(np.float32)
    B = workloads.lowrank(n, n, sig, seed + 1).astype(np.float32)
    return A, B


def test_estimate_matches_oracle_and_exact(L):
    from paper_2405_16917_gb300 import tune
    A, B = _operands(512, 61)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    plan = L.Plan(512, 512, 512, 48, 8, 1, seed=7, prec=(1, 1, 2), sketch=L.SKETCH_TF32)
    D = L.matmul(plan, At, Bt)
    est = tune.estimate_error(At, Bt, D, probes=16, seed=5)
    G = tune.probe_matrix(512, 16, 5).cpu().numpy()
    Dn = D.cpu().numpy()
    ref = oracle.tune.probe_error(A, B, Dn, G)
    assert abs(est - ref) <= 1e-4 * ref, (est, ref)
    exact = oracle.lramm.rel_fro(Dn, oracle.lramm.exact_product(A, B))
    assert abs(est - exact) <= 0.25 * exact, (est, exact)


def test_tune_choice(L):
    from paper_2405_16917_gb300 import tune
    A, B = _operands(768, 62)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    target = 0.06
    choice, cands = tune.tune(At, Bt, target, ranks=[32, 96], triples=("888", "884", "444"), probes=16)
    assert len(cands) == 6
    assert choice == oracle.tune.select(cands, target)
    # the chosen configuration's exact error is within the estimate's accuracy of the target
    plan = L.Plan(768, 768, 768, choice["r"], 16, 1, seed=7, prec=tune.TRIPLES[choice["triple"]],
                  sketch=L.SKETCH_TF32)
    D = L.matmul(plan, At, Bt).cpu().numpy()
    exact = oracle.lramm.rel_fro(D, oracle.lramm.exact_product(A, B))
    if choice["err"] <= target:
        assert exact <= 1.25 * target, (choice, exact)
    # a larger rank with the same bits is at least as accurate (estimates, 25% slack)
    by = {(c["r"], c["triple"]): c for c in cands}
    for t in ("888", "884", "444"):
        assert by[(96, t)]["err"] <= 1.25 * by[(32, t)]["err"]
