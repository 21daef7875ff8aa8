"""Write tests/golden/oracle_values.npz from the oracle alone.

Values: FP64 oracle results on the seeded workloads at their stated sizes,
used by the GPU parity tests (the oracle is too slow to rerun there):
  two_layer_direct     direct sum, two-layer N=1000, all targets
  three_layer_sel      sampled target indices, three-layer N=32768
  three_layer_direct   direct sum at those targets
  three_layer_fmm      oracle FMM (p=8, leaf 64) at those targets
Run:  python tests/golden/make_golden.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fmm, green  # noqa: E402
from oracle.media import Medium  # noqa: E402
from paper_1902_05132_gb300 import workloads  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.npz")


def main():
    res = {}
    t = time.time()
    w = workloads.two_layer()
    med = Medium(w["k"], w["d"], w["eps"])
    res["two_layer_direct"] = green.direct_sum(med, w["src"], w["q"], w["tgt"])
    print("two-layer direct", time.time() - t, flush=True)
    w = workloads.three_layer()
    med = Medium(w["k"], w["d"], w["eps"])
    sel = workloads.sample_targets(len(w["tgt"]), 24, seed=11)
    res["three_layer_sel"] = sel
    t = time.time()
    res["three_layer_direct"] = green.direct_sum(med, w["src"], w["q"], w["tgt"], targets=sel)
    print("three-layer direct", time.time() - t, flush=True)
    t = time.time()
    res["three_layer_fmm"] = fmm.FMM(med, w["p"], w["leaf"]).evaluate(w["src"], w["q"], w["tgt"], targets=sel)
    print("three-layer fmm", time.time() - t, flush=True)
    np.savez_compressed(OUT, **res)


if __name__ == "__main__":
    main()
