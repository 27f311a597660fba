"""Survey of the coagulation tests (Appendix A, B) on the GPU: W1 distance to the
Smoluchowski solution over neighbourhood sizes N_K and interval tolerances eps.

    python tests/coag_survey.py [--n 1000000] [--seeds 1] [--nk 256] [--eps 0.08]
                                [--kernels constant,linear,product]

Per run: N_p equal-mass particles with unit grains (gamma(2) grains for the linear
kernel) in a periodic unit box, V_i = 1, the library's mixed form, evolved to the final
t~ of the kernel (constant 1e8, linear 4, product 0.9: Appendix B).  The constant and
linear runs are one bounded collision step (gd_collide) over the whole time: the
particles do not move, so the neighbour lists are built once and every later interval
only refreshes the partner snapshot.  The product runs permute the particle positions
before every interval's neighbour build (the paper's reshuffle of the cached lists,
Appendix B).  Prints one JSON line per (kernel, N_K, eps) with W1 (dex) averaged over
the seeds, its spread, the intervals and the wall time per run.
"""
import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from paper_2609_35967_gb300 import workloads as W  # noqa: E402

import coag_exact as X  # noqa: E402

T_END = {"constant": 1e8, "linear": 4.0, "product": 0.9}
MODE = {"constant": W.CONSTANT, "linear": W.LINEAR, "product": W.PRODUCT}


def run(gd, kernel, n, nk, eps, seed):
    import torch
    t_end = T_END[kernel]
    ins = W.coag_instance(n, K=nk, mode=MODE[kernel], seed=seed, eps=eps, dt_coll=t_end)
    sess = gd.Session([ins], precision=gd.GD_MIXED)
    rng = np.random.default_rng(5000 + seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if kernel == "product":
        t = 0.0
        n_iv = 0
        while t < t_end * (1.0 - 1e-12):
            # a finite-sampling runaway gels the system early and the intervals shrink to
            # dt_coll / 2^60: stop there (reported) rather than loop on ever shorter intervals
            n_iv += 1
            if n_iv > 20000:
                break
            p = torch.as_tensor(rng.permutation(n), device=sess.device)
            for k in ("x", "y", "z"):
                sess.t[k].copy_(sess.t[k][p].clone())
            torch.cuda.synchronize()     # the library's stream reads the permuted positions
            sess.build_neighbors()
            sess.collision_rates()
            sess.sample_collisions()
            st_now = sess.stats(check=False)
            t += st_now["instances"][0]["dt_exe"]
            if st_now["status"]:
                break
    else:
        sess.collide(t_end)
        t = t_end
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    st = sess.stats(check=False)
    s = sess.t["s"].cpu().numpy()
    sess.close()
    m = math.pi * ins["params"]["rho_s"] * s ** 3 / 6.0
    cdf, lo = {"constant": (X.cdf_constant, 0.0), "linear": (X.cdf_linear, -3.0),
               "product": (X.cdf_product, 0.0)}[kernel]
    w = X.w1(m, ins["M"], cdf(t), lo, math.log10(max(m.max(), 10.0)) + 0.5)
    mean = {"constant": X.mean_constant, "linear": X.mean_linear, "product": X.mean_product}[kernel](t)
    # mass-weighted mean grain mass (equal particle masses) against the moment equation
    return w, el, st["intervals"], st["status"], float(np.sum(ins["M"] * m) / np.sum(ins["M"])) / mean, t


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1000000)
    ap.add_argument("--seeds", type=int, default=1)
    ap.add_argument("--nk", default="256")
    ap.add_argument("--eps", default="0.08")
    ap.add_argument("--kernels", default="constant,linear,product")
    args = ap.parse_args()
    from paper_2609_35967_gb300 import binding as gd
    gd.load()
    for kernel in args.kernels.split(","):
        for nk in (int(v) for v in args.nk.split(",")):
            for eps in (float(v) for v in args.eps.split(",")):
                ws, els, ivs, mrs, stops = [], [], [], [], []
                for seed in range(args.seeds):
                    w, el, iv, status, mr, t = run(gd, kernel, args.n, nk, eps, 100 + seed)
                    if status != 0 or t < T_END[kernel] * (1.0 - 1e-9):
                        stops.append({"seed": 100 + seed, "status": status, "t": t})
                        continue
                    ws.append(w)
                    els.append(el)
                    ivs.append(iv)
                    mrs.append(mr)
                line = {"kernel": kernel, "N_K": nk, "eps": eps, "n": args.n, "seeds": args.seeds,
                        "t_end": T_END[kernel]}
                if ws:
                    line.update({"W1": float(np.mean(ws)), "W1_sd": float(np.std(ws)),
                                 "mean_ratio": float(np.mean(mrs)), "intervals": float(np.mean(ivs)),
                                 "s_per_run": float(np.mean(els))})
                if stops:
                    line["stopped_early"] = stops    # runaway growth before t_end (product kernel)
                print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
