"""Write the stored expected values of the full-size Munk workload (N = 4095, 2000 steps of
50 m, [6/6] Pade, Neumann to 1e-10 or 12 terms, f = 50 Hz, source at 1000 m) by running the
FP64 oracle only.  Output: munk_n4095_s2000.txt (sampled final field and TL rows).

    python tests/golden/make_golden.py            # several minutes on a multi-core host
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import sssp_oracle as O  # noqa: E402
from paper_2511_03343_gb300 import inputs  # noqa: E402

FIELD_STRIDE = 4      # every 4th depth point of the final field
TL_EVERY = 100        # TL rows after steps 100, 200, ..., 2000
TL_STRIDE = 16        # every 16th depth point of those rows


def main(path=os.path.join(HERE, "munk_n4095_s2000.txt")):
    s = inputs.munk()
    g = O.Grid(N=s.N, H=s.H, k0=s.k0, dr=s.dr)
    t0 = time.time()
    res = O.march(s.u0, s.profiles, g, s.pade_order, s.steps, s.neumann_terms, s.neumann_tol,
                  tl_every=TL_EVERY)
    el = time.time() - t0
    idx = np.arange(0, s.N, FIELD_STRIDE)
    tidx = np.arange(0, s.N, TL_STRIDE)
    with open(path, "w") as f:
        f.write("# FP64 oracle (sum form, Algorithm 1), written by tests/golden/make_golden.py\n")
        f.write(f"# munk N={s.N} H={s.H} f={s.freq} dr={s.dr} steps={s.steps} p={s.pade_order} "
                f"terms={s.neumann_terms} tol={s.neumann_tol} zs={s.zs} c0={s.c0} oracle_seconds={el:.1f}\n")
        f.write(f"field_stride {FIELD_STRIDE} tl_every {TL_EVERY} tl_stride {TL_STRIDE} norm {np.linalg.norm(res.u):.17e}\n")
        f.write("field\n")
        for i in idx:
            f.write(f"{i} {res.u[i].real:.17e} {res.u[i].imag:.17e}\n")
        f.write("tl\n")
        for r, row in zip(res.tl_ranges, res.tl):
            f.write(f"{r:.6f} " + " ".join(f"{row[i]:.10e}" for i in tidx) + "\n")
    print("wrote", path, "in", round(el, 1), "s")


def load(path=os.path.join(HERE, "munk_n4095_s2000.txt")):
    lines = open(path).read().splitlines()
    hdr = lines[2].split()
    meta = {hdr[k]: float(hdr[k + 1]) for k in range(0, len(hdr), 2)}
    fi = lines.index("field")
    ti = lines.index("tl")
    field_idx, field = [], []
    for ln in lines[fi + 1:ti]:
        a = ln.split()
        field_idx.append(int(a[0]))
        field.append(float(a[1]) + 1j * float(a[2]))
    tl_r, tl = [], []
    for ln in lines[ti + 1:]:
        a = ln.split()
        tl_r.append(float(a[0]))
        tl.append([float(v) for v in a[1:]])
    return meta, np.array(field_idx), np.array(field), np.array(tl_r), np.array(tl)


if __name__ == "__main__":
    main()
