"""Writes the oracle's expected values for the two full-size 3D workloads.

TEST INFRASTRUCTURE.  Calls only oracle/ (FP64 NumPy) on the seeded inputs of
synth/; nothing here comes from the CUDA path.  The full-size GPU parity tests
(tests/test_gpu_full_size.py) read these files, because the oracle needs hours
of host time for what the GPU does in seconds:

* full_peg_in_bore_3d_rho.npz, full_docking_2000_500_rho.npz
    rho (Eq. 13/15/16c/17t, complex FP64) at every query point of both shapes,
    with the sample counts and input fingerprints they were computed from.
* full_peg_in_bore_3d_rotations.txt
    for every one of the 576 Hopf rotations, the band-limited periodic score map
    Re f_N(R, t) on the 128^3 grid (direct nonuniform DFT, spectral product,
    inverse FFT, with weights c = rho v): its maximum, the flat index of the
    maximum (lowest on ties), the second-largest value, max |Re f_N| and max |f_N|.
* full_peg_in_bore_3d_top10.txt
    the global top-10 over those per-rotation maxima (score desc, rotation asc,
    index asc) and the continuous score f_c (Eq. 8 for Gaussian-represented
    SDFs, FP64 pair sums over all pairs) at each of the ten poses.

Run from the repository root (hours on a few cores; resumable):
    python tests/golden/make_full_size.py [--workers 8] [--only peg|docking]
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import score as oscore  # noqa: E402
from oracle import sdf as osdf  # noqa: E402
from synth import configs  # noqa: E402

RHO_CHUNK = 256        # query points per oracle call
FC_SLICE = 1024        # moving samples per oracle call (f_c is a sum over them)


def fingerprint(s):
    """Sums that identify a shape's generated inputs (counts and positions)."""
    return np.array([s.boundary.pos.shape[0], s.query.pos.shape[0], s.boundary.pos.sum(), s.query.pos.sum(),
                     s.boundary.area.sum(), s.query.vol.sum()])


def rho_all(s, params, pool):
    p, b = s.query.pos, s.boundary
    parts = list(pool.map(lambda lo: osdf.sdf_rho(p[lo:lo + RHO_CHUNK], b.pos, b.normal, b.area, **params),
                          range(0, len(p), RHO_CHUNK)))
    return np.concatenate(parts)


def rho_file(w, pool):
    path = os.path.join(HERE, f"full_{w.name}_rho.npz")
    if os.path.exists(path):
        d = np.load(path)
        return d["rho_fixed"], d["rho_moving"]
    t0 = time.time()
    r1 = rho_all(w.fixed, w.sdf_params(), pool)
    r2 = rho_all(w.moving, w.sdf_params(), pool)
    np.savez_compressed(path, rho_fixed=r1, rho_moving=r2, fp_fixed=fingerprint(w.fixed),
                        fp_moving=fingerprint(w.moving))
    print(f"{path}: {time.time() - t0:.0f} s", flush=True)
    return r1, r2


def f_c(p1, c1, p2, c2, q, t, sigma_g, pool):
    parts = pool.map(lambda lo: oscore.pair_score_fc(p1, c1, p2[lo:lo + FC_SLICE], c2[lo:lo + FC_SLICE], q, t,
                                                     sigma_g, chunk=256),
                     range(0, len(p2), FC_SLICE))
    return sum(parts)


def peg(pool):
    w = configs.peg_in_bore_3d()
    r1, r2 = rho_file(w, pool)
    p1, c1 = w.fixed.query.pos, osdf.sdf_weights(r1, w.fixed.query.vol)
    p2, c2 = w.moving.query.pos, osdf.sdf_weights(r2, w.moving.query.vol)
    path = os.path.join(HERE, f"full_{w.name}_rotations.txt")
    part = path + ".partial"
    done = {}
    if os.path.exists(part):
        for line in open(part):
            if line.strip() and not line.startswith("#"):
                v = line.split()
                done[int(v[0])] = line
    if not os.path.exists(path):
        F1 = oscore.nudft(p1, c1, w.N, w.L, -1)
        with open(part, "a") as f:
            for r in range(w.n_rot):
                if r in done:
                    continue
                t0 = time.time()
                m = oscore.score_map_fN(p1, c1, p2, c2, w.quats[r], w.N, w.L, w.sigma_g, F1=F1)
                re = m.real.ravel()
                best, idx = oscore.rotation_best(m.real)
                second = np.partition(re, -2)[-2]
                line = (f"{r} {best!r} {int(idx)} {float(second)!r} {float(np.abs(re).max())!r} "
                        f"{float(np.abs(m).max())!r}\n")
                f.write(line)
                f.flush()
                done[r] = line
                print(f"rotation {r}: {time.time() - t0:.1f} s", flush=True)
        with open(path, "w") as f:
            f.write("# rot best_re_fN argmax_flat_index second_re_fN max_abs_re_fN max_abs_fN "
                    "(peg_in_bore_3d, 128^3, oracle weights c = rho v)\n")
            for r in range(w.n_rot):
                f.write(done[r])
        os.remove(part)
    rows = np.loadtxt(path)
    top_path = os.path.join(HERE, f"full_{w.name}_top10.txt")
    if not os.path.exists(top_path):
        top = oscore.global_top_k(rows[:, 1], rows[:, 2].astype(int), 10)
        with open(top_path, "w") as f:
            f.write("# rank rot argmax_flat_index re_fN re_fc im_fc (FP64 pair sums over all pairs)\n")
            for k, (r, s, i) in enumerate(top):
                t = oscore.translation_of_index(i, w.N, w.L, 3)
                t0 = time.time()
                fc = f_c(p1, c1, p2, c2, w.quats[r], t, w.sigma_g, pool)
                f.write(f"{k} {r} {i} {float(s)!r} {float(fc.real)!r} {float(fc.imag)!r}\n")
                f.flush()
                print(f"f_c rank {k}: {time.time() - t0:.0f} s", flush=True)


def docking(pool):
    rho_file(configs.docking_2000_500(), pool)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    ap.add_argument("--only", choices=["peg", "docking"], default=None)
    a = ap.parse_args()
    with cf.ThreadPoolExecutor(a.workers) as pool:
        if a.only in (None, "docking"):
            docking(pool)
        if a.only in (None, "peg"):
            peg(pool)


if __name__ == "__main__":
    main()
