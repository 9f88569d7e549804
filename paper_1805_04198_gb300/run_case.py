"""Runs the solver once on a named synthetic workload and prints its statistics.

Meant for profilers and quick checks: the inputs are generated on the host,
copied to the device, and one solve is enqueued and waited for.

  python -m paper_1805_04198_gb300.run_case --workload dd4097 [--max-iter K] [--theta T] [--dtype f32|f64]
  python -m paper_1805_04198_gb300.run_case --workload fsm4097
  python -m paper_1805_04198_gb300.run_case --workload dd3d257 [--max-iter K] [--theta T]
  python -m paper_1805_04198_gb300.run_case --workload batch256 [--nprob P] [--max-iter K]

dd4097   4097^2 Fourier-mode slowness, left-edge source, 16x16 subdomains,
         coarse ratio 16 (the benchmark's DD workload), weight --theta
         (default 0.2, the weight the kernel profiles were taken with; the
         benchmark itself uses 0)
fsm4097  the same grid solved by the plain full-grid FSM
dd3d257  257^3 point source, 8^3 subdomains, coarse ratio 8 (the 3-D workload)
batch256 mixed-size batch (sides 257..2049, 8..32 subdomains per side)
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import eik, inputs


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", required=True, choices=["dd4097", "fsm4097", "dd3d257", "batch256"])
    ap.add_argument("--max-iter", type=int, default=None)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--nprob", type=int, default=256)
    ap.add_argument("--n", type=int, default=4097)
    ap.add_argument("--theta", type=float, default=0.2)
    a = ap.parse_args(argv)
    npd = np.float32 if a.dtype == "f32" else np.float64
    dev = torch.device("cuda", 0)
    eik.load()
    if a.workload == "dd3d257":
        w = inputs.workload_c2()
        r = torch.from_numpy(w["r"].astype(npd)).to(dev)
        gm = torch.from_numpy(w["gamma"]).to(dev)
        g = torch.from_numpy(w["g"].astype(npd)).to(dev)
        k = a.max_iter if a.max_iter is not None else w["max_iter"]
        u, st = eik.dd_solve(r, gm, g, w["h"], w["tiles"], w["c"], theta=a.theta, max_iter=k, tol=0.0,
                             max_coarse_sweeps=8)
        torch.cuda.synchronize()
        print(json.dumps(st))
        return
    if a.workload in ("dd4097", "fsm4097"):
        w = inputs.workload_c1(n=a.n)
        r = torch.from_numpy(w["r"].astype(npd)).to(dev)
        gm = torch.from_numpy(w["gamma"]).to(dev)
        g = torch.from_numpy(w["g"].astype(npd)).to(dev)
        if a.workload == "fsm4097":
            u, st = eik.fsm(r, gm, g, w["h"])
        else:
            k = a.max_iter if a.max_iter is not None else w["max_iter"]
            u, st = eik.dd_solve(r, gm, g, w["h"], w["tiles"], w["c"], theta=a.theta, max_iter=k, tol=1e-6,
                                 max_coarse_sweeps=8)
        torch.cuda.synchronize()
        print(json.dumps(st))
        return
    probs = []
    for q in inputs.workload_c3(nprob=a.nprob):
        probs.append(dict(r=torch.from_numpy(q["r"].astype(npd)).to(dev), gamma=torch.from_numpy(q["gamma"]).to(dev),
                          g=torch.from_numpy(q["g"].astype(npd)).to(dev), h=q["h"], tiles=q["tiles"],
                          coarse_ratio=q["c"], theta=q["theta"],
                          max_iter=q["max_iter"] if a.max_iter is None else min(a.max_iter, q["max_iter"]),
                          tol=q["tol"]))
    B = eik.DDBatch(probs)
    B.run()
    torch.cuda.synchronize()
    st = B.stats()
    print(json.dumps({"nprob": len(st), "fine_updates": sum(s["fine_updates"] for s in st),
                      "coarse_updates": sum(s["coarse_updates"] for s in st), "launches": st[0]["launches"]}))


if __name__ == "__main__":
    main()
