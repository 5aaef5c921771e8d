"""Precision sweep of LRAMM against the direct quantised products (the
paper's Fig. 3 study, Sec. 4.2): relative Frobenius error against the FP64
product for i.i.d. uniform, exponential, normal and binary entries, ranks
from dim/20 to dim/2, bit-width triples (d1 d2 d3) and plain FP32 factors,
next to DQ8 and DQ4 on the same operands.

  python -m paper_2405_16917_gb300.sweep [--n 1024] [--p 16] [--q 1] [--out sweep.json]

Prints one JSON line per (distribution, method, rank) and a markdown table.
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

import workloads  # noqa: E402

TRIPLES = {"884": (1, 1, 2), "844": (1, 2, 2), "444": (2, 2, 2), "888": (1, 1, 1), "float": (0, 0, 0)}


def main(argv=None):
    import torch

    import paper_2405_16917_gb300 as L

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--p", type=int, default=16)
    ap.add_argument("--q", type=int, default=1)
    ap.add_argument("--dists", default=",".join(workloads.ENTRY_DISTS))
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    n = args.n
    dev = torch.device("cuda", 0)
    L.load()
    # ranks from dim/20 to dim/2 (l = r + p a multiple of 4: the blocked Cholesky's layout)
    ranks = sorted({max(4, (n // d) // 4 * 4 - args.p % 4) for d in (20, 10, 5, 4, 3)} | {n // 2 - args.p})
    rows = []
    for di, dist in enumerate(args.dists.split(",")):
        A = torch.from_numpy(workloads.entry_matrix(dist, n, n, 2001 + di).astype(np.float32)).to(dev)
        B = torch.from_numpy(workloads.entry_matrix(dist, n, n, 3001 + di).astype(np.float32)).to(dev)
        exact = A.double() @ B.double()
        nrm = exact.norm().item()

        def err(D):
            return ((D.double() - exact).norm() / nrm).item()

        for name, pq in (("DQ8", 1), ("DQ4", 2)):
            rows.append({"dist": dist, "method": name, "r": n, "err": err(L.dq_matmul(A, B, prec=pq))})
        for r in ranks:
            for tname, prec in TRIPLES.items():
                plan = L.Plan(n, n, n, r, args.p, args.q, seed=workloads.SEED_SKETCH, prec=prec,
                              sketch=L.SKETCH_F32 if tname == "float" else L.SKETCH_TF32)
                ws = plan.workspace(dev)
                D = L.matmul(plan, A, B, ws=ws)
                st = L.status_read(ws)
                rows.append({"dist": dist, "method": "LRAMM(%s)" % tname, "r": r, "err": err(D), "status": st})
                del plan, ws, D
        for row in rows:
            if row["dist"] == dist:
                print(json.dumps(row))
        sys.stdout.flush()
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"n": n, "p": args.p, "q": args.q, "rows": rows}, f)
    # markdown: one table per distribution, methods x ranks
    for dist in args.dists.split(","):
        sub = [x for x in rows if x["dist"] == dist]
        dq = {x["method"]: x["err"] for x in sub if x["method"].startswith("DQ")}
        print("\n%s entries (n = %d, p = %d, q = %d): DQ8 %.3g, DQ4 %.3g" % (dist, n, args.p, args.q, dq["DQ8"],
                                                                        dq["DQ4"]))
        print("| method | " + " | ".join("r = %d" % r for r in ranks) + " |")
        print("|---|" + "---|" * len(ranks))
        for tname in TRIPLES:
            m = "LRAMM(%s)" % tname
            vals = {x["r"]: x["err"] for x in sub if x["method"] == m}
            print("| %s | " % m + " | ".join("%.3g" % vals[r] for r in ranks) + " |")
    return 0


if __name__ == "__main__":
    sys.exit(main())
