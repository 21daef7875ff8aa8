"""Write tests/golden/oracle_values_full.npz from the oracle alone.

Values (FP64 oracle results on the seeded workloads at their stated sizes,
used by the GPU parity tests and reported by the benchmark; the oracle is
too slow to rerun there):
  three_layer_sel2000     2,000 sampled target indices, three-layer N=32,768
  three_layer_direct2000  direct sum at those targets
  three_layer_fmm_sel     200 of them (the first 200 of a second sample)
  three_layer_fmm200      oracle FMM (p=8, leaf 64) at those targets
  three_layer_1m_sel      128 sampled targets of the three-layer N=1,048,576
                          workload with complex charges (p=10)
  three_layer_1m_direct   direct sum at those targets
The direct sums run in worker processes (spawn), a slice of targets each.
Run:  python tests/golden/make_golden_full.py [workers]
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values_full.npz")


def _direct_part(args):
    n, complex_charges, p, idx = args
    sys.path.insert(0, ROOT)
    from oracle import green
    from oracle.media import Medium
    from paper_1902_05132_gb300 import workloads
    w = workloads.three_layer(n=n, p=p, complex_charges=complex_charges)
    med = Medium(w["k"], w["d"], w["eps"])
    return green.direct_sum(med, w["src"], w["q"], w["tgt"], targets=idx)


def _fmm_part(args):
    idx, = args
    sys.path.insert(0, ROOT)
    from oracle import fmm
    from oracle.media import Medium
    from paper_1902_05132_gb300 import workloads
    w = workloads.three_layer()
    med = Medium(w["k"], w["d"], w["eps"])
    return fmm.FMM(med, w["p"], w["leaf"]).evaluate(w["src"], w["q"], w["tgt"], targets=idx)


def _parallel(pool, n, complex_charges, p, sel, parts):
    chunks = np.array_split(sel, parts)
    res = pool.map(_direct_part, [(n, complex_charges, p, c) for c in chunks])
    return np.concatenate(res)


def main():
    from paper_1902_05132_gb300 import workloads
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else max(1, os.cpu_count() - 1)
    res = {}
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        t = time.time()
        fmm_sel = workloads.sample_targets(32768, 200, seed=21)
        fmm_job = pool.map_async(_fmm_part, [(fmm_sel,)])
        sel = workloads.sample_targets(32768, 2000, seed=20)
        res["three_layer_sel2000"] = sel
        res["three_layer_direct2000"] = _parallel(pool, 32768, False, 8, sel, 4 * workers)
        print("three-layer direct at 2000 targets", time.time() - t, flush=True)
        t = time.time()
        sel1m = workloads.sample_targets(1048576, 128, seed=22)
        res["three_layer_1m_sel"] = sel1m
        res["three_layer_1m_direct"] = _parallel(pool, 1048576, True, 10, sel1m, 2 * workers)
        print("N=2^20 direct at 128 targets", time.time() - t, flush=True)
        res["three_layer_fmm_sel"] = fmm_sel
        res["three_layer_fmm200"] = fmm_job.get()[0]
        print("three-layer oracle FMM at 200 targets done", flush=True)
    np.savez_compressed(OUT, **res)


if __name__ == "__main__":
    main()
