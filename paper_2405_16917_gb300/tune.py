"""Parameter tuning of LRAMM (Sec. 3.5): the rank r and the bit widths
(d1, d2, d3) for a target relative Frobenius error, by measurement.

Sec. 3.5 relates the running time to r and the bit widths and recommends r
near a tenth of the dimension with d2 = 4, d1 = d3 = 8.  Here every
candidate (r, triple) runs on the device: its time is measured with CUDA
events and its error against A B estimated with s Gaussian probe columns G
(n x s): e = ||(A B - D) G||_F / ||A B G||_F, with E ||X G||_F^2 = s ||X||_F^2,
so A B is never formed (A (B G) and D G are FP32 products of the library).
The choice is the fastest candidate whose estimated error is at most the
target, else the most accurate one.

  python -m paper_2405_16917_gb300.tune [--n 2048] [--target 0.05]

Every product runs in the library on the current CUDA device.
"""
import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

I8, I4 = 1, 2
TRIPLES = {"888": (I8, I8, I8), "884": (I8, I8, I4), "848": (I8, I4, I8), "844": (I8, I4, I4),
           "444": (I4, I4, I4)}
PROBE_STREAM = 2   # Philox stream of the probe matrix (Omega_A and Omega_B use 0 and 1)


def probe_matrix(n, probes, seed):
    """G (n x probes): the library's Philox Gaussian, stream 2."""
    import paper_2405_16917_gb300 as L
    return L.gaussian(seed, PROBE_STREAM, n, probes)


def estimate_error(A, B, D, probes=8, seed=11):
    """||(A B - D) G||_F / ||A B G||_F with G = n x probes Gaussian (FP32 products).

    The products run in the library; the two Frobenius norms of the m x
    probes results are taken on the host.  They are the tuner's measurement
    of a candidate's error (a few thousand numbers), not a step of the
    product path, which lramm_matmul runs entirely on the device."""
    import paper_2405_16917_gb300 as L
    n = B.shape[1]
    G = probe_matrix(n, probes, seed)
    BG = L.sketch_product(B, G, sketch=L.SKETCH_F32)
    ABG = L.sketch_product(A, BG, sketch=L.SKETCH_F32)
    DG = L.sketch_product(D, G, sketch=L.SKETCH_F32)
    abg = ABG.double().cpu().numpy()
    dg = DG.double().cpu().numpy()
    return float(np.linalg.norm(abg - dg) / np.linalg.norm(abg))


MAX_L = 544   # the SVD form's largest sketch (r + p)


def candidate_ranks(m, n, k, p):
    """Ranks around a tenth of the smallest dimension: dim/40 .. dim/5, multiples
    of 4, within the SVD form's sketch limit (r + p <= 544)."""
    dim = min(m, n, k)
    out = []
    for div in (40, 20, 10, 5):
        r = max(4, (dim // div) // 4 * 4)
        r = min(r, (MAX_L - p) // 4 * 4)
        if r + p <= dim and r not in out:
            out.append(r)
    return out


def tune(A, B, target, ranks=None, triples=tuple(TRIPLES), p=16, q=1, seed=7, probes=8, reps=3):
    """Measure every (r, triple) candidate and return (choice, candidates);
    each candidate is a dict with r, triple, ms (median device time of one
    lramm_matmul) and err (probe estimate)."""
    import torch

    import paper_2405_16917_gb300 as L
    m, k = A.shape
    n = B.shape[1]
    ranks = ranks or candidate_ranks(m, n, k, p)
    out = torch.empty((m, n), dtype=torch.float32, device=A.device)
    cands = []
    for r in ranks:
        for name in triples:
            plan = L.Plan(m, n, k, r, p, q, seed=seed, prec=TRIPLES[name], sketch=L.SKETCH_TF32)
            ws = plan.workspace(A.device)
            L.matmul(plan, A, B, out=out, ws=ws)
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                L.matmul(plan, A, B, out=out, ws=ws)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            st = L.status_read(ws)
            if st not in (0, 7):
                raise L.LrammError(st, "tune: r=%d %s" % (r, name))
            cands.append(dict(r=r, triple=name, ms=float(np.median(ts)),
                              err=estimate_error(A, B, out, probes=probes)))
    ok = [c for c in cands if c["err"] <= target]
    choice = min(ok, key=lambda c: (c["ms"], c["err"])) if ok else min(cands, key=lambda c: c["err"])
    return choice, cands


def main(argv=None):
    import torch

    import workloads

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--target", type=float, default=0.05)
    ap.add_argument("--spectrum", default="poly1")
    args = ap.parse_args(argv)
    n = args.n
    sig = workloads.spectrum(args.spectrum, n)
    A = torch.from_numpy(workloads.lowrank(n, n, sig, workloads.SEED_A).astype(np.float32)).cuda()
    B = torch.from_numpy(workloads.lowrank(n, n, sig, workloads.SEED_B).astype(np.float32)).cuda()
    choice, cands = tune(A, B, args.target)
    for c in cands:
        print(json.dumps(c))
    print(json.dumps({"choice": choice, "target": args.target, "n": n, "spectrum": args.spectrum}))


if __name__ == "__main__":
    sys.exit(main())
