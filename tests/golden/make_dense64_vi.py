"""Write tests/golden/dense64_vi_samples.npz: the FP64 oracle's value
iteration of the 4-D dense CP model 64^4 (8 actions, rank 8, gamma 0.95,
seed 0) from V = 0 to max|V' - V| < 1e-6, sampled at 4096 seeded states.

Calls only oracle/ (dense.value_iteration, dense.q_values) and the shared
input generator; nothing here comes from the CUDA path. Each oracle sweep
at this size is a few hundred FP64 tensordot products over 16.8M states
(tens of seconds on a multi-core host), so the full solve takes an hour or
more: run it once and commit the output.

    python tests/golden/make_dense64_vi.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import cpmdp_inputs as ci  # noqa: E402
from oracle import dense as od  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dense64_vi_samples.npz")
NSAMPLE = 4096
TOL = 1e-6


def main():
    dc = ci.config_dense_4d(side=64, seed=0)
    t0 = time.time()
    V = np.zeros(dc.nstates)
    trace = []
    k = 0
    while True:
        k += 1
        Q = od.q_values(dc, V)
        Vn = Q.max(axis=0)
        res = float(np.max(np.abs(Vn - V)))
        trace.append(res)
        V = Vn
        print(f"sweep {k}: residual {res:.6e} ({time.time() - t0:.0f} s)", flush=True)
        if res < TOL or k >= 1000:
            break
    # greedy policy of the returned V, its Q gaps, and the oracle's own
    # certified residual max |T(V) - V|
    Q = od.q_values(dc, V)
    TV = Q.max(axis=0)
    cert = float(np.max(np.abs(TV - V)))
    Qs = np.sort(Q, axis=0)
    gap = Qs[-1] - Qs[-2]
    pi = Q.argmax(axis=0).astype(np.uint8)
    idx = np.unique((ci.u64(0, 99, NSAMPLE) % np.uint64(dc.nstates)).astype(np.int64))
    np.savez_compressed(OUT, state=idx, value=V[idx], policy=pi[idx], gap=gap[idx], sweeps=k,
                        residual=res, certified_residual=cert, max_abs_value=float(np.abs(V).max()),
                        mean_value=float(V.mean()), trace=np.asarray(trace))
    print(f"wrote {OUT}: {k} sweeps, residual {res:.3e}, certified {cert:.3e}, "
          f"{time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
