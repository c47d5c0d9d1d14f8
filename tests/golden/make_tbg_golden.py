"""Write cached FP64 oracle values for the full-size parity tests.

Calls only the oracle (``oracle/``) and the seeded input generators
(``synth``); nothing here touches the CUDA path.  Output:
``tests/golden/tbg_oracle_samples.npz`` holding, for twisted bilayer graphene
m = 29 (10,444 atoms, 1512 x 1512 x 281 grid, the benchmark's workload):

  h_keys (n_blocks, 5)   pattern blocks (I, J, t1, t2, t3) drawn at random, plus on-site blocks
  h_vals (sum nw_I nw_J) their H^V values (Eq. 2), row-major, back to back
  r_idx  (n_points, 3)   grid points drawn inside the bilayer (|z - layer centre| within 3.5 bohr
                          of the layers), where rho is non-zero
  r_vals (n_points,)     rho at those points (Eq. 3)
  f_atoms, f_vals, f_vir  8 random atoms: F_I and the per-atom virial Pi_I (Eq. 4, 5)

and for m = 5 (364 atoms) the full per-atom virial, hence the stress
sigma = -sum_I Pi_I / Omega, and every force (m5_F, m5_vir, m5_sigma).

Inputs: V = 16 seeded plane waves (seed 2), D = seeded symmetric density matrix on the
pattern (seed 3), exactly as the tests and the benchmark build them.

Usage:  python tests/golden/make_tbg_golden.py [--blocks 1000] [--points 10000] [--atoms 8]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "tbg_oracle_samples.npz")


def layer_band(s, half_width=3.5):
    """Grid indices along a3 whose plane lies within half_width bohr of a layer."""
    n3 = s.grid[2]
    c = s.cell[2, 2]
    z = np.arange(n3) * c / n3
    zl = np.unique(np.round(s.pos[:, 2], 6))
    keep = np.zeros(n3, bool)
    for z0 in zl:
        keep |= np.abs(z - z0) <= half_width
    return np.nonzero(keep)[0]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--blocks", type=int, default=1000)
    ap.add_argument("--points", type=int, default=10000)
    ap.add_argument("--atoms", type=int, default=8)
    ap.add_argument("--m5", type=int, default=5, help="TBG index of the full-stress cell")
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    rng = np.random.default_rng(2409)
    t0 = time.time()
    s = synth.tbg(29)
    o = oracle.Oracle(s)
    print(f"m=29 oracle pattern: {len(o.blocks)} blocks ({time.time() - t0:.0f} s)", flush=True)
    V = synth.v_grid(s.grid, synth.plane_wave_params()).numpy()
    D = o.d_fill()
    print(f"inputs ready ({time.time() - t0:.0f} s)", flush=True)
    blocks = o.blocks
    onsite = np.nonzero((blocks[:, 0] == blocks[:, 1]) & (blocks[:, 2:] == 0).all(1))[0]
    sel = np.concatenate([rng.choice(len(blocks), args.blocks - 16, replace=False),
                          rng.choice(onsite, 16, replace=False)])
    keys = blocks[sel]
    t1 = time.time()
    H = o.vlocal_blocks(V, keys)
    print(f"{len(keys)} H blocks ({time.time() - t1:.0f} s)", flush=True)
    band = layer_band(s)
    idx = np.stack([rng.integers(0, s.grid[0], args.points), rng.integers(0, s.grid[1], args.points),
                    rng.choice(band, args.points)], 1).astype(np.int64)
    t1 = time.time()
    rho = o.rho_points(D, idx)
    print(f"{len(idx)} rho points ({time.time() - t1:.0f} s); zero: {np.mean(rho == 0):.3f}", flush=True)
    atoms = rng.choice(s.n_atoms, args.atoms, replace=False).astype(np.int64)
    t1 = time.time()
    F, W = o.force(V, D, atoms=atoms)
    print(f"{len(atoms)} atoms ({time.time() - t1:.0f} s)", flush=True)
    del V, D, o
    s5 = synth.tbg(args.m5)
    o5 = oracle.Oracle(s5)
    V5 = synth.v_grid(s5.grid, synth.plane_wave_params()).numpy()
    D5 = o5.d_fill()
    t1 = time.time()
    F5, W5 = o5.force(V5, D5)
    sigma5 = -W5.sum(0) / o5.omega
    print(f"m={args.m5}: all {s5.n_atoms} atoms ({time.time() - t1:.0f} s)", flush=True)
    np.savez_compressed(args.out, h_keys=keys.astype(np.int32), h_vals=np.concatenate([h.reshape(-1) for h in H]),
                        r_idx=idx.astype(np.int32), r_vals=rho, f_atoms=atoms.astype(np.int32), f_vals=F,
                        f_vir=W, m5=np.int32(args.m5), m5_F=F5, m5_vir=W5, m5_sigma=sigma5)
    print(f"wrote {args.out} ({os.path.getsize(args.out) / 1e6:.2f} MB, {time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
