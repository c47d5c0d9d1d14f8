#!/usr/bin/env python
"""Benchmark: grid points per second of real-space grid integration (gint).

One step = gint_vlocal (H^V, Eq. 2) + gint_rho (rho, Eq. 3) + gint_force_stress
(Pulay force and stress, Eq. 4-5) over the whole grid of one synthetic
twisted-bilayer-graphene cell (default: m = 29, 10,444 C atoms,
1512 x 1512 x 281 = 6.42e8 grid points, C DZP basis, rc = 7 bohr).
value = grid points x steps / time (all ranks).  Inputs stay resident in HBM
during the timed steps; V (5.1 GB) and rho (5.1 GB) exceed L2, so no flush is
needed between steps.

Each call takes the cheapest tensor-core form that meets its stated error
(H <= 1e-7 Ha, rho <= 1e-6 normwise, F <= 1e-5 Ha/bohr): the exact form
(fp16x4) for H^V and rho, the three-product form (fp16x3) for the force
(--precision picks one form for all calls, or one per call).

--impl reference times the FP64 oracle (oracle/, plain C + OpenMP) on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (description, tbg index m)
    "tbg_m29": ("twisted bilayer graphene m=29, 10444 C atoms, DZP, rc 7 bohr, h=pi/20 bohr", 29),
    "tbg_m15": ("twisted bilayer graphene m=15, 2884 C atoms, DZP, rc 7 bohr, h=pi/20 bohr", 15),
    "tbg_m10": ("twisted bilayer graphene m=10, 1324 C atoms, DZP, rc 7 bohr, h=pi/20 bohr", 10),
    "tbg_m5": ("twisted bilayer graphene m=5, 364 C atoms, DZP, rc 7 bohr, h=pi/20 bohr", 5),
}
DEFAULT_FORMS = "vlocal=fp16x4,rho=fp16x4,force=fp16x3"
METRIC = "grid pts/s for gint H^V+rho(+force), mixed vs FP64 form at stated error, TBG 10,444"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = sorted(float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit())
        mx = max((float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """x of this rank -> the largest x over the ranks (x itself for one rank)."""
    if ws == 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, ws, t_max_ms):
    """Units that all ranks processed in the timed steps, per second of the slowest rank."""
    return units_per_rank * steps * ws / (t_max_ms / 1e3)


# ----------------------------------------------------------------- oracle arm
def oracle_inputs(system):
    """The oracle and its inputs for `system` (input generation and set-up, never timed)."""
    import oracle
    import synth
    o = oracle.Oracle(system)
    V = synth.v_grid(system.grid, synth.plane_wave_params()).numpy()
    D = o.d_fill()
    return o, V, D


def oracle_sample(system, n_points, n_blocks, n_atoms_f, seed=11, inputs=None):
    """Time the FP64 oracle on a bounded random sample and scale to the whole step.

    Returns (seconds for one full step as extrapolated, description, sampled
    oracle outputs).  rho: n_points random grid points (uniform over the grid, so
    vacuum included); H: n_blocks random pattern blocks; force: n_atoms_f random
    atoms.  Each part is scaled by (total / sampled).
    """
    import numpy as np
    rng = np.random.default_rng(seed)
    o, V, D = inputs if inputs is not None else oracle_inputs(system)
    idx = np.stack([rng.integers(0, system.grid[i], n_points) for i in range(3)], 1)
    t0 = time.perf_counter()
    rho_s = o.rho_points(D, idx)
    t_rho = time.perf_counter() - t0
    bsel = rng.choice(len(o.blocks), size=min(n_blocks, len(o.blocks)), replace=False)
    keys = o.blocks[bsel]
    t0 = time.perf_counter()
    H_s = o.vlocal_blocks(V, keys)
    t_h = time.perf_counter() - t0
    atoms = rng.choice(system.n_atoms, size=min(n_atoms_f, system.n_atoms), replace=False)
    t0 = time.perf_counter()
    F_s, _ = o.force(V, D, atoms=atoms)
    t_f = time.perf_counter() - t0
    full = (t_rho * system.n_grid / n_points + t_h * len(o.blocks) / len(keys)
            + t_f * system.n_atoms / len(atoms))
    desc = {"rho_points": int(n_points), "h_blocks": int(len(keys)), "force_atoms": int(len(atoms)),
            "sample_seconds": t_rho + t_h + t_f,
            "scaled": "each part scaled by total/sampled (grid points, pattern blocks, atoms)"}
    samples = {"idx": idx, "rho": rho_s, "blocks": bsel, "H": H_s, "atoms": atoms, "F": F_s,
               "oracle_blocks": o.blocks}
    return full, desc, samples


def oracle_sample_parts(system, n_points, n_blocks, inputs, seed=17):
    """Seconds the oracle takes for n_points rho points and n_blocks H blocks (a fixed sample)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    o, V, D = inputs
    idx = np.stack([rng.integers(0, system.grid[i], n_points) for i in range(3)], 1)
    keys = o.blocks[rng.choice(len(o.blocks), size=min(n_blocks, len(o.blocks)), replace=False)]
    t0 = time.perf_counter()
    o.rho_points(D, idx)
    o.vlocal_blocks(V, keys)
    return time.perf_counter() - t0, f"{n_points} rho points and {len(keys)} H blocks"


CALLS = ("vlocal", "rho", "force")
TC_PRODUCTS = {"fp16x3": 3, "bf16x3": 3, "fp16x4": 6}  # 16-bit tensor products per credited product
DTYPES = {"fp64": "f64", "fp32": "f32", "fp16x3": "f16x3", "bf16x3": "bf16x3", "fp16x4": "f16x4"}


def parse_forms(spec):
    """'fp16x4' (every call) or 'vlocal=fp16x4,rho=fp16x4,force=fp16x3' (one form per call)."""
    if "=" not in spec:
        return {c: spec for c in CALLS}
    forms = {}
    for item in spec.split(","):
        k, v = item.split("=")
        if k not in CALLS:
            raise SystemExit(f"--precision: unknown call {k!r} (expected one of {CALLS})")
        forms[k] = v
    if set(forms) != set(CALLS):
        raise SystemExit(f"--precision: give a form for each of {CALLS}")
    return forms


def launches_per_step(forms):
    """Kernels of ours per step: the call's kernel, plus the mirror (and, exact form, the
    normalisation) after H^V; the D row maxima (exact form) and D format before the
    tensor-core rho and force kernels; the empty-brick fill after rho; the finalize after force."""
    tc = lambda f: f in TC_PRODUCTS  # noqa: E731
    ex = lambda f: f == "fp16x4"  # noqa: E731
    n = 2 + ex(forms["vlocal"])
    n += 2 + tc(forms["rho"]) + ex(forms["rho"])
    n += 2 + tc(forms["force"]) + ex(forms["force"])
    return int(n)


def sample_errors(samples, H, rho, F, blocks, offsets):
    """Errors of GPU results against the oracle's sampled outputs (same pattern order)."""
    import numpy as np
    if not np.array_equal(blocks, samples["oracle_blocks"]):
        return {"error": "pattern differs from the oracle's"}
    Hn = H.cpu().numpy()
    eh = 0.0
    for b, ref in zip(samples["blocks"], samples["H"]):
        eh = max(eh, float(np.max(np.abs(Hn[offsets[b]:offsets[b + 1]].reshape(ref.shape) - ref))))
    idx = samples["idx"]
    rho_g = rho[idx[:, 0], idx[:, 1], idx[:, 2]].cpu().numpy()
    er = float(np.max(np.abs(rho_g - samples["rho"])) / max(1e-300, np.max(np.abs(samples["rho"]))))
    ef = float(np.max(np.abs(F.cpu().numpy()[samples["atoms"]] - samples["F"])))
    return {"H_abs": eh, "rho_rel": er, "F_abs": ef, "gates": {"H_abs": 1e-7, "rho_rel": 1e-6, "F_abs": 1e-5}}


GOLDEN = os.path.join(ROOT, "tests", "golden", "tbg_oracle_samples.npz")


def block_keys(blocks):
    """One int64 per pattern block (I, J, t1, t2, t3), increasing with the pattern's sort order."""
    import numpy as np
    b = np.asarray(blocks, dtype=np.int64)
    return ((((b[:, 0] << 14) + b[:, 1]) * 64 + b[:, 2] + 32) * 64 + b[:, 3] + 32) * 64 + b[:, 4] + 32


def golden_errors(H, rho, F, blocks, offsets, path=GOLDEN):
    """Errors against the cached FP64 oracle values of the TBG m=29 cell (written by
    tests/golden/make_tbg_golden.py): H on its sampled blocks (max abs), rho at its points inside
    the bilayer (normwise), F of its atoms (max abs)."""
    import numpy as np
    z = np.load(path)
    keys = block_keys(z["h_keys"])
    allk = block_keys(blocks)
    pos = np.searchsorted(allk, keys)
    if np.any(pos >= len(allk)) or np.any(allk[np.minimum(pos, len(allk) - 1)] != keys):
        return {"error": "a cached block is missing from the pattern"}
    Hn = H.cpu().numpy()
    vals = z["h_vals"]
    eh, o = 0.0, 0
    for b in pos:
        n = int(offsets[b + 1] - offsets[b])
        eh = max(eh, float(np.max(np.abs(Hn[offsets[b]:offsets[b + 1]] - vals[o:o + n]))))
        o += n
    idx = z["r_idx"].astype(np.int64)
    rg = rho[idx[:, 0], idx[:, 1], idx[:, 2]].cpu().numpy()
    er = float(np.max(np.abs(rg - z["r_vals"])) / np.max(np.abs(z["r_vals"])))
    ef = float(np.max(np.abs(F.cpu().numpy()[z["f_atoms"].astype(np.int64)] - z["f_vals"])))
    return {"H_abs": eh, "rho_rel": er, "F_abs": ef, "gates": {"H_abs": 1e-7, "rho_rel": 1e-6, "F_abs": 1e-5},
            "sample": f"cached oracle values: {len(keys)} blocks, {len(idx)} points inside the bilayer, "
                      f"{len(z['f_atoms'])} atoms"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    name = args.workload
    desc, m = WORKLOADS[name]
    system = synth.tbg(m)
    cores = oracle.num_threads()
    step_times = []
    sample = None
    inputs = oracle_inputs(system)
    for i in range(args.warmup + args.steps):
        t_full, sample, _ = oracle_sample(system, args.ref_points, args.ref_blocks, args.ref_atoms, seed=100 + i,
                                          inputs=inputs)
        if i >= args.warmup:
            step_times.append(t_full)
    t = sum(step_times) / len(step_times)
    value = system.n_grid / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "grid_points/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "description": desc, "grid": list(system.grid),
                       "grid_points": system.n_grid, "atoms": system.n_atoms,
                       "precision": "fp64 (the oracle, plain C + OpenMP on the host cores)"},
            "cpu_baseline": {"value": value, "unit": "grid_points/s", "cores": cores, "kind": "oracle",
                             "sample": json.dumps(sample)},
            "e2e": {"value": value, "unit": "grid_points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- our arm
class EndToEnd:
    """Steps through the public API with the inputs in pinned host memory: every step copies V
    and D to the device, runs H^V, rho and force/stress, and copies H, rho, F, sigma and E back.

    ``use(call)`` sets the handle's form for a call (or does nothing).  ``inline`` keeps the
    copies in line with each step on the compute stream; ``overlapped`` hides them behind the
    neighbouring steps' compute (uploads of step k + 1 and downloads of step k on two copy
    streams, ordered by events, with two sets of device inputs and outputs)."""

    def __init__(self, g, V, D, use, stream, dev):
        import torch
        self.g, self.use, self.stream, self.dev = g, use, stream, dev
        self.Vh = V.cpu().pin_memory()
        self.Dh = D.cpu().pin_memory()
        n_at = g.n_atoms
        f64 = torch.float64
        self.Hh = torch.empty(g.n_values, dtype=f64).pin_memory()
        self.rhoh = torch.empty(g.grid, dtype=f64).pin_memory()
        self.Fh = torch.empty((n_at, 3), dtype=f64).pin_memory()
        self.sigh = torch.empty((3, 3), dtype=f64).pin_memory()
        self.Eh = torch.empty(1, dtype=f64).pin_memory()

        def outs():
            return (torch.empty(g.n_values, dtype=f64, device=dev), torch.empty(g.grid, dtype=f64, device=dev),
                    torch.empty((n_at, 3), dtype=f64, device=dev), torch.empty((3, 3), dtype=f64, device=dev),
                    torch.empty((n_at, 3, 3), dtype=f64, device=dev), torch.empty(1, dtype=f64, device=dev))
        self.Vd = [torch.empty_like(V), None]
        self.Dd = [torch.empty_like(D), None]
        self.out = [outs(), None]
        self._outs = outs
        self.h2d_bytes = (self.Vh.numel() + self.Dh.numel()) * 8
        self.d2h_bytes = (self.Hh.numel() + self.rhoh.numel() + self.Fh.numel() + self.sigh.numel()
                          + self.Eh.numel()) * 8

    def _compute(self, j):
        H, rho, F, sig, vir, E = self.out[j]
        self.use("vlocal")
        self.g.vlocal(self.Vd[j], H, stream=self.stream)
        self.use("rho")
        self.g.rho(self.Dd[j], rho, stream=self.stream)
        self.use("force")
        self.g.force_stress(self.Vd[j], self.Dd[j], out=(F, sig, vir, E), stream=self.stream)

    def _download(self, j):
        H, rho, F, sig, _, E = self.out[j]
        self.Hh.copy_(H, non_blocking=True)
        self.rhoh.copy_(rho, non_blocking=True)
        self.Fh.copy_(F, non_blocking=True)
        self.sigh.copy_(sig, non_blocking=True)
        self.Eh.copy_(E, non_blocking=True)

    def step(self):
        """One step with its copies on the compute stream."""
        import torch
        with torch.cuda.stream(self.stream):
            self.Vd[0].copy_(self.Vh, non_blocking=True)
            self.Dd[0].copy_(self.Dh, non_blocking=True)
            self._compute(0)
            self._download(0)

    def inline(self, n):
        """ms per step of n steps with the copies in line."""
        import torch
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(self.stream)
        for _ in range(n):
            self.step()
        b.record(self.stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    def overlapped(self, n):
        """ms per step of n steps with overlapped copies, from the first upload to the last download."""
        import torch
        ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        if self.Vd[1] is None:
            self.Vd[1], self.Dd[1], self.out[1] = torch.empty_like(self.Vd[0]), torch.empty_like(self.Dd[0]), self._outs()
        st = self.stream
        cin, cout = torch.cuda.Stream(device=self.dev), torch.cuda.Stream(device=self.dev)
        ev_in, ev_done, ev_out = [ev(), ev()], [ev(), ev()], [ev(), ev()]
        start, stop = ev(), ev()
        start.record(st)
        cin.wait_event(start)
        with torch.cuda.stream(cin):
            self.Vd[0].copy_(self.Vh, non_blocking=True)
            self.Dd[0].copy_(self.Dh, non_blocking=True)
        ev_in[0].record(cin)
        for k in range(n):
            j = k & 1
            st.wait_event(ev_in[j])
            if k >= 2:
                st.wait_event(ev_out[j])  # the outputs of step k - 2 have been read back
            self._compute(j)
            ev_done[j].record(st)
            if k + 1 < n:
                if k >= 1:
                    cin.wait_event(ev_done[1 - j])  # step k - 1 no longer reads inputs 1 - j
                with torch.cuda.stream(cin):
                    self.Vd[1 - j].copy_(self.Vh, non_blocking=True)
                    self.Dd[1 - j].copy_(self.Dh, non_blocking=True)
                ev_in[1 - j].record(cin)
            cout.wait_event(ev_done[j])
            with torch.cuda.stream(cout):  # one copy stream: downloads into the host buffers stay in order
                self._download(j)
            ev_out[j].record(cout)
        st.wait_event(ev_out[(n - 1) & 1])
        stop.record(st)
        torch.cuda.synchronize()
        return start.elapsed_time(stop) / n


def run_ours(args):
    import numpy as np
    import torch

    import synth
    from paper_2409_09399_gb300 import gint

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    desc, m = WORKLOADS[args.workload]
    system = synth.tbg(m)
    ng = system.n_grid
    forms = parse_forms(args.precision)
    prec = forms["vlocal"]
    mixed_forms = len(set(forms.values())) > 1
    torch.cuda.synchronize()
    t_setup0 = time.perf_counter()
    g = gint.from_system(system, precision=prec, brick=tuple(args.brick), device=local)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup0  # pattern, binning, tables: once per geometry
    info = g.info()
    V = synth.v_grid(system.grid, synth.plane_wave_params(), device=dev)
    blocks, offsets = g.pattern()
    D = synth.d_fill_torch(blocks, offsets[:-1], g.n_values, system.pos, system.cell, system.nw(), dev)
    H = torch.empty(g.n_values, dtype=torch.float64, device=dev)
    rho = torch.empty(system.grid, dtype=torch.float64, device=dev)
    F = torch.empty((system.n_atoms, 3), dtype=torch.float64, device=dev)
    sig = torch.empty((3, 3), dtype=torch.float64, device=dev)
    vir = torch.empty((system.n_atoms, 3, 3), dtype=torch.float64, device=dev)
    E = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    n_ev = 4

    def use(call):
        # the form of each call (a host-side field of the handle; no device work)
        if mixed_forms:
            g.set_precision(forms[call])

    def step(record=None):
        if record is not None:
            record[0].record(stream)
        use("vlocal")
        g.vlocal(V, H, stream=stream)
        if record is not None:
            record[1].record(stream)
        use("rho")
        g.rho(D, rho, stream=stream)
        if record is not None:
            record[2].record(stream)
        use("force")
        g.force_stress(V, D, out=(F, sig, vir, E), stream=stream)
        if record is not None:
            record[3].record(stream)

    for _ in range(args.warmup):
        step()
    g.sync()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    recs = [[ev() for _ in range(n_ev)] for _ in range(args.steps)]
    end = ev()
    barrier()
    with ClockSampler(local) as clocks:
        t0 = ev()
        t0.record(stream)
        for k in range(args.steps):
            step(recs[k])
        end.record(stream)
        torch.cuda.synchronize()
    barrier()
    g.sync()
    total_ms = t0.elapsed_time(end)
    parts = np.zeros(3)
    for k in range(args.steps):
        r = recs[k]
        parts += [r[0].elapsed_time(r[1]), r[1].elapsed_time(r[2]), r[2].elapsed_time(r[3])]
    parts /= args.steps
    t_max = max_over_ranks(total_ms, ws, dev)
    ms_per_step = t_max / args.steps
    value = whole_job_rate(ng, args.steps, ws, t_max)

    H_mixed, rho_mixed, F_mixed = H.clone(), rho.clone(), F.clone()

    # ---- FP64 form on the same GPU (one step, same inputs)
    fp64 = None
    if args.fp64_steps > 0 and set(forms.values()) != {"fp64"}:
        saved, mixed_saved = dict(forms), mixed_forms
        forms.update({c: "fp64" for c in CALLS})
        mixed_forms = False
        g.set_precision("fp64")
        step()
        g.sync()
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.fp64_steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        g.sync()
        ms64 = a.elapsed_time(b) / args.fp64_steps
        fp64 = {"value": ng / (ms64 / 1e3), "unit": "grid_points/s", "ms_per_step": ms64,
                "speedup_of_mixed": ms64 / ms_per_step}
        H_fp64, rho_fp64, F_fp64 = H.clone(), rho.clone(), F.clone()
        forms.update(saved)
        mixed_forms = mixed_saved
        g.set_precision(prec)

    # ---- end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        runner = EndToEnd(g, V, D, use, stream, dev)
        runner.step()
        torch.cuda.synchronize()
        barrier()
        ms_one = runner.overlapped(args.e2e_steps) if args.e2e_overlap else runner.inline(args.e2e_steps)
        barrier()
        g.sync()
        ms_e2e = max_over_ranks(ms_one, ws, dev)
        e2e = {"value": whole_job_rate(ng, 1, ws, ms_e2e), "unit": "grid_points/s",
               "h2d_bytes_per_step": runner.h2d_bytes, "d2h_bytes_per_step": runner.d2h_bytes, "ms_per_step": ms_e2e,
               "copies": "overlapped with the neighbouring steps" if args.e2e_overlap else "in line with the step"}
        del runner

    # ---- the local potential from rho (Hartree by FFT + LDA XC), the step that feeds V back into
    #      H^V; timed on its own, outside the metric's step
    local_pot = None
    if args.local_potential_steps > 0:
        Vo = torch.empty_like(rho)
        en = g.local_potential(rho, V_out=Vo)[2]
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(args.local_potential_steps):
            g.local_potential(rho, V_out=Vo, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms_lp = a.elapsed_time(b) / args.local_potential_steps
        local_pot = {"ms_per_call": ms_lp, "grid_points_per_s": ng / (ms_lp / 1e3),
                     "includes": "two 3-D FFTs (cuFFT, a library step), the G-space Hartree multiply and the "
                                 "fused LDA pass with FP64 energies", "E_H": float(en[0]), "E_xc": float(en[1])}
        del Vo

    # ---- roofline of the dominant call
    peaks, peak_src = load_peaks()
    sum_no, sum_no2 = g.work_stats()
    flops = {"vlocal": float(sum_no2 + sum_no), "rho": float(sum_no2 + sum_no),
             "force": float(2 * sum_no2 + 24 * sum_no)}
    names = ["vlocal", "rho", "force"]
    dom = int(np.argmax(parts))
    dom_name = names[dom]
    achieved = flops[dom_name] / (parts[dom] / 1e3) / 1e12
    dom_prec = forms[dom_name]
    if dom_prec == "fp64":
        peak, bound, src = 1.25, "alu", "FP64 1.25 TFLOP/s nominal (DFMA; recipe table)"
    elif dom_prec == "fp32":
        peak, bound = 152 * 128 * 2 * 2.07e9 / 1e12, "alu"
        src = "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
    else:
        # fp16 and bf16 share the dense 16-bit tensor rate
        peak, bound = peaks.get("bf16_tflops_sustained", 1711.1), "tensor"
        src = f"16-bit dense tensor, sustained ({peak_src} bf16 cuBLAS loop)"
    traffic = None
    tpath = os.path.join(ROOT, "profiles", f"traffic_{dom_name}_{dom_prec}.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        # DRAM bytes from an ncu capture, valid only while the kernel sources it was taken on are unchanged
        import hashlib
        hs = hashlib.sha256()
        for path in tj.get("sources", []):
            with open(os.path.join(ROOT, path), "rb") as f:
                hs.update(f.read())
        if tj.get("workload_scaled_to", tj.get("scaled_to", {}).get("workload")) == args.workload and \
                hs.hexdigest() == tj.get("source_sha256"):
            traffic = tj.get("bytes_per_launch")
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": dom_name, "peak_source": src,
            "algorithmic_flop_per_launch": flops[dom_name]}
    # split forms issue k 16-bit products per credited product: the fraction against peak / k
    k_products = TC_PRODUCTS.get(dom_prec)
    if k_products:
        roof["products_per_flop"] = k_products
        roof["frac_of_peak_over_products"] = achieved / (peak / k_products)

    # ---- CPU baseline (oracle, bounded sample), rank 0 at N = 1 only
    cpu = None
    errors = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        inputs = oracle_inputs(system)
        t_full, sample, samples = oracle_sample(system, args.ref_points, args.ref_blocks, args.ref_atoms,
                                                inputs=inputs)
        cores = oracle.num_threads()
        cpu = {"value": ng / t_full, "unit": "grid_points/s", "cores": cores, "kind": "oracle",
               "sample": json.dumps(sample)}
        # one thread: a smaller sample of rho points and H blocks; the force part is scaled from the
        # all-core force time by the one-thread / all-core ratio of the other two parts
        if args.ref_points_1thread > 0:
            oracle.set_num_threads(1)
            try:
                t1, s1 = oracle_sample_parts(system, args.ref_points_1thread, args.ref_blocks_1thread, inputs)
            finally:
                oracle.set_num_threads(cores)
            tN, _ = oracle_sample_parts(system, args.ref_points_1thread, args.ref_blocks_1thread, inputs)
            ratio = t1 / tN
            cpu["one_thread"] = {"value": ng / (t_full * ratio), "unit": "grid_points/s", "cores": 1,
                                 "sample": f"{s1}; one-thread / {cores}-thread time ratio {ratio:.2f} on that "
                                           "sample, applied to the whole all-core step estimate"}
        errors = {args.precision: sample_errors(samples, H_mixed, rho_mixed, F_mixed, blocks, offsets)}
        if fp64 is not None:
            errors["fp64"] = sample_errors(samples, H_fp64, rho_fp64, F_fp64, blocks, offsets)
        errors["sample"] = "oracle outputs at the cpu_baseline sample (random points, blocks, atoms)"
        if args.workload == "tbg_m29" and os.path.exists(GOLDEN):
            errors["cached"] = {args.precision: golden_errors(H_mixed, rho_mixed, F_mixed, blocks, offsets)}
            if fp64 is not None:
                errors["cached"]["fp64"] = golden_errors(H_fp64, rho_fp64, F_fp64, blocks, offsets)

    gb = lambda n: f"{n * 8 / 1e9:.1f} GB"  # noqa: E731
    l2_note = (f"inputs larger than L2 (V {gb(ng)}, rho {gb(ng)}, D {gb(g.n_values)})" if ng * 8 > 256e6 else
               f"V {gb(ng)}, rho {gb(ng)}, D {gb(g.n_values)}: not larger than L2 (profiling / test size)")
    line = {"metric": METRIC, "value": value, "unit": "grid_points/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ",".join(dict.fromkeys(DTYPES.get(forms[c], forms[c]) for c in CALLS)),
            "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "grid": list(system.grid),
                       "grid_points": ng, "atoms": system.n_atoms,
                       "precision": forms if mixed_forms else prec,
                       "brick": list(info["brick"]), "l2": l2_note,
                       "parallelism": "replicas" if ws > 1 else "single", "setup_s": t_setup},
            "ms_per_call": {"vlocal": parts[0], "rho": parts[1], "force_stress": parts[2]},
            "fp64_form": fp64, "errors_vs_oracle": errors, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
            "local_potential": local_pot,
            "clocks": clocks.summary(), "gpu_launches": launches_per_step(forms) * args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """The uneven multi-cell workload: random C/H/O cells in one batched launch per step."""
    import numpy as np
    import torch

    import synth
    from paper_2409_09399_gb300.batch import GintBatch
    n_cells = int(args.workload[len("batch"):])
    torch.cuda.set_device(0)
    systems = [synth.random_cell(i) for i in range(n_cells)]
    t0 = time.perf_counter()
    b = GintBatch(systems, precision=args.precision, brick="auto",
                  candidates=((8, 8, 8), (4, 8, 8), (4, 4, 8), (4, 4, 4), (3, 3, 4), (2, 2, 4), (2, 2, 2)),
                  sample=4)
    t_setup = time.perf_counter() - t0
    Vs, Ds, Hs, rhos, Fs, sigs, Es = [], [], [], [], [], [], []
    for s_, h in zip(systems, b.handles):
        blocks, offsets = h.pattern()
        Vs.append(synth.v_grid(s_.grid, synth.plane_wave_params(), device="cuda"))
        Ds.append(synth.d_fill_torch(blocks, offsets[:-1], h.n_values, s_.pos, s_.cell, s_.nw(), "cuda"))
        Hs.append(torch.empty(h.n_values, dtype=torch.float64, device="cuda"))
        rhos.append(torch.empty(h.grid, dtype=torch.float64, device="cuda"))
        Fs.append(torch.empty((h.n_atoms, 3), dtype=torch.float64, device="cuda"))
        sigs.append(torch.empty((3, 3), dtype=torch.float64, device="cuda"))
        Es.append(torch.empty(1, dtype=torch.float64, device="cuda"))
    for _ in range(args.warmup):
        b.run(Vs, Ds, Hs, rhos, Fs, sigs, Es)
    torch.cuda.synchronize()
    for h in b.handles:
        h.sync()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        a.record()
        for _ in range(args.steps):
            b.run(Vs, Ds, Hs, rhos, Fs, sigs, Es)
        e.record()
        torch.cuda.synchronize()
    ms = a.elapsed_time(e) / args.steps
    pts = int(sum(np.prod(s_.grid) for s_ in systems))
    shapes = {}
    for br in b.bricks:
        shapes[str(tuple(br))] = shapes.get(str(tuple(br)), 0) + 1
    line = {"metric": f"grid pts/s for gint H^V+rho(+force), {n_cells} uneven C/H/O cells in one batched launch",
            "value": pts / (ms / 1e3), "unit": "grid_points/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": args.workload, "cells": n_cells, "grid_points": pts,
                       "atoms": int(sum(s_.n_atoms for s_ in systems)), "precision": args.precision,
                       "bricks": shapes, "autotuner_ranking": [list(r) for r in (b.ranking or [])],
                       "setup_s": t_setup, "queue": "one launch per call over the (cell, brick) queue"},
            "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch256", "batch64"], default="tbg_m29")
    ap.add_argument("--precision", default=None,
                    help=f"one form for every call, or one per call (default {DEFAULT_FORMS}; batches: fp16x4)")
    ap.add_argument("--brick", type=int, nargs=3, default=[0, 0, 0])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--local-potential-steps", type=int, default=3)
    ap.add_argument("--e2e-inline", dest="e2e_overlap", action="store_false",
                    help="keep each step's host copies in line with its compute (default: overlap them with the "
                         "neighbouring steps' compute on two copy streams)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-points", type=int, default=2000)
    ap.add_argument("--ref-blocks", type=int, default=24)
    ap.add_argument("--ref-atoms", type=int, default=1)
    ap.add_argument("--ref-points-1thread", type=int, default=400)
    ap.add_argument("--ref-blocks-1thread", type=int, default=6)
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp16x4" if args.workload.startswith("batch") else DEFAULT_FORMS
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.workload.startswith("batch"):
        if "=" in args.precision:
            raise SystemExit("--precision: the batched workload takes one form for every call")
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no oracle timing arm"}))
            return 0
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
