#!/usr/bin/env python
"""Throughput of the batched RGF hot path on GB300.

One step = the whole path over one batch: lead self-energies (OBC), the fused
G^R + G^< forward/backward sweeps, and the observables (T, DOS, current,
density), for 1024 energy points of the ballistic nb = 64, b = 128 device
(S = I + 0.05 R).  ``value`` is energy points per second for the whole job
(all ranks), inputs resident in HBM; ``e2e`` repeats it through host buffers.
With torchrun (N > 1) every rank solves its own 1024 energies (weak scaling,
no data-path collective: energies are independent).

``--impl reference`` times the CPU oracle (numpy complex128) on a bounded
sample of the same workload instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

# BF16 slice-pair products per complex product in the sliced GEMM: NS (NS + 1) / 2 for NS
# digits per value (s + t <= NS + 1); set from the loaded library by run_gpu
OZ_SLICE_PAIRS = 36.0

METRIC = ("energy points/sec (G^R+G^< RGF, nb=64, bs=128) mixed vs FP64 on 1 GB300 at ≤1e-6 rel")
UNIT = "energy points/s"


# ---------------------------------------------------------------------------
# helpers (host logic; covered by CPU tests)
# ---------------------------------------------------------------------------

def rank_energies(ne_per_rank, rank, world, e_min=-3.0, e_max=3.0):
    """Energies of one rank: the global grid of ne_per_rank*world points,
    interleaved so that every rank sees the same spread of in-band and
    out-of-band energies."""
    grid = np.linspace(e_min, e_max, ne_per_rank * world)
    return grid[rank::world].copy()


def rank_weights(ne_per_rank, rank, world, e_min=-3.0, e_max=3.0):
    """Quadrature weights of one rank's energies: the trapezoid weights of the global
    grid (ne_per_rank*world points) taken at this rank's points, so that the ranks'
    weighted partial sums add up to the integral over the whole grid."""
    grid = np.linspace(e_min, e_max, ne_per_rank * world)
    return W.trapezoid_weights(grid)[rank::world].copy()


def sum_over_ranks(t, world):
    """In-place sum of a tensor over the ranks (the energy integral's exchange step)."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def energy_integrals(density, current, T, fL, fR, w, ne, nb, world):
    """The energy-integrated observables of the whole grid, summed over the ranks (each
    rank's density output is already its weighted sum): the total density, the
    interface currents I_i = sum_E w(E) J_i(E) at the first and the last interface, and
    the Landauer current sum_E w(E) T(E) (f_L - f_R).  In a ballistic device the
    interface currents differ from one another only by the eta sink of the blocks
    between them (Sec. III's conservation check holds up to O(eta))."""
    cur = sum_over_ranks((w.view(ne, 1) * current.view(ne, nb - 1)).sum(0), world)
    dens = sum_over_ranks(density.sum().reshape(1).clone(), world)
    land = sum_over_ranks((w * T * (fL - fR)).sum().reshape(1), world)
    return {"collective": f"all_reduce sum over {world} ranks" if world > 1 else "none (one rank)",
            "density_total": float(dens.item()), "current_interface_first": float(cur[0].item()),
            "current_interface_last": float(cur[-1].item()), "current_landauer": float(land.item())}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def max_over_ranks(x, world, device=None):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def roofline_for(cls, stats, peaks, peak_src, sustained=True):
    """Roofline object for one kernel class from live event timings.

    gemm_oz, gemm_tc : complex block products on the tensor cores.  achieved =
              useful complex flops (8 n^3 per product) / time; peak = the useful peak
              of a complex product on the tensor cores, TF32 dense peak / 3 (a complex
              product costs 24 n^3 TF32 flops as a 3-term split), the TF32 peak taken as
              the bf16 peak x (1.1 / 2.25) (nominal ratio).  For the sliced product the
              executed BF16 work (OZ_SLICE_PAIRS x useful) against the bf16 peak is
              reported beside it (tensor-pipe occupancy by the emulation).
    gemm_f64, inv_f64: FP64 pipe ("alu"), peak 1.25 TFLOP/s nominal.
    inv_f32 : FP32 CUDA cores ("alu"), peak 152 SM x 128 lanes x 2 x 2.07 GHz."""
    ms = stats["ms"]
    fl = stats["flops"]
    n = max(stats["launches"], 1)
    per_launch_s = ms / 1e3 / n
    achieved = (fl / n) / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    bf16 = peaks["bf16_tflops_sustained" if sustained else "bf16_tflops"]
    extra = {}
    if cls == "gemm_oz":
        bound, peak, unit = "tensor", bf16 * (1.1 / 2.25) / 3.0, "TFLOP/s"
        note = (f"useful complex flops (8 n^3 per product) vs TF32 peak/3 (TF32 = bf16 "
                f"{'sustained' if sustained else 'burst'} {peak_src} x 1.1/2.25)")
        extra = {"executed_bf16_tflops": achieved * OZ_SLICE_PAIRS,
                 "executed_bf16_frac": achieved * OZ_SLICE_PAIRS / bf16,
                 "executed_note": f"{OZ_SLICE_PAIRS:.0f} BF16 slice-pair products per complex product "
                                  f"vs bf16 {'sustained' if sustained else 'burst'} {peak_src} peak"}
    elif cls == "gemm_tc":
        bound, peak, unit = "tensor", bf16 * (1.1 / 2.25) / 3.0, "TFLOP/s"
        note = f"useful complex flops vs TF32 peak/3 (TF32 = bf16 {peak_src} x 1.1/2.25)"
    elif cls in ("gemm_f64", "inv_f64"):
        bound, peak, unit = "alu", 1.25, "TFLOP/s"
        note = "FP64 pipe, nominal 1.25 TFLOP/s"
    elif cls == "inv_f32":
        bound, peak, unit = "alu", 152 * 128 * 2 * 2.07e9 / 1e12, "TFLOP/s"
        note = "FP32 CUDA cores, 152 SM x 128 x 2 x 2.07 GHz"
    else:
        bound, peak, unit = "hbm", peaks["hbm_gbs"], "GB/s"
        achieved = (stats["bytes"] / n) / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
        note = f"HBM ({peak_src})"
    useful = (fl / n) / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    out = {"kernel": cls, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
           "useful_tflops": useful,
           "frac": achieved / peak if peak else None, "launches": stats["launches"],
           "avg_launch_ms": ms / n, "peak_source": f"{peak_src}: {note}"}
    out.update(extra)
    return out


def traffic_record(cls):
    """The committed ncu record of the kernel class (bytes and duration of one full
    launch), or None when that capture does not match the current kernel source."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    ent = d.get(cls)
    if not ent:
        return None
    src = os.path.join(ROOT, ent["source"])
    if not os.path.exists(src):
        return None
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    if h != ent.get("source_sha256_16"):
        return None
    return ent


def traffic_for(cls):
    """Per-launch DRAM traffic of the kernel class from the committed ncu summary,
    or None when that capture does not match the current kernel source."""
    ent = traffic_record(cls)
    return ent.get("bytes_per_launch_full") if ent else None


def hbm_for(cls, peaks, peak_src):
    """Achieved DRAM bandwidth of one full launch of the kernel class (the ncu record's
    bytes over its durations) against the HBM peak, or None without a current record."""
    ent = traffic_record(cls)
    if not ent or not ent.get("ms_per_launch_full"):
        return None
    gbs = ent["bytes_per_launch_full"] / (ent["ms_per_launch_full"] / 1e3) / 1e9
    return {"achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"],
            "note": f"ncu DRAM bytes / duration of one full launch vs HBM copy peak ({peak_src})"}


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------

def oracle_step(dev, idx, weights):
    """The whole path for energies ``idx`` with the CPU oracle: OBC, the block
    recursion for G^R and G^< (pinned to dense inversion by the tests), T, DOS,
    current and the weighted density contribution."""
    from oracle import negf_oracle as O
    n = np.zeros(dev.nb * dev.b)
    for e in idx:
        out = O.solve_energy(dev, int(e), lesser=True, use_rgf=True)
        n += weights[e] * out["n_E"]
    return n


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return int(max(i.get("num_threads", 1) for i in info))
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_baseline(dev, budget_s=15.0, min_energies=2):
    """Times the oracle on a bounded, spread-out sample of the workload's energies."""
    w = dev.weights()
    order = np.random.default_rng(0).permutation(dev.ne)
    t0 = time.perf_counter()
    done = 0
    for e in order:
        oracle_step(dev, [e], w)
        done += 1
        if done >= min_energies and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{done} of {dev.ne} energies of the nb={dev.nb}, b={dev.b} device "
                      f"(OBC + block RGF G^R/G^< + observables, numpy complex128), {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    dev = W.config2(nb=args.nb, b=args.b, ne=args.ne)
    w = dev.weights()
    rng = np.random.default_rng(1)
    per = args.ref_energies
    for _ in range(args.warmup):
        oracle_step(dev, rng.choice(dev.ne, per, replace=False), w)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(dev, rng.choice(dev.ne, per, replace=False), w)
    dt = time.perf_counter() - t0
    val = per * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"config 2: ballistic batched RGF, nb={args.nb}, b={args.b}, "
                                   f"{args.ne} energies in [-3,3], S=I+0.05R; each step {per} sampled energies",
                       "nb": args.nb, "b": args.b, "energies": args.ne},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{per} random energies per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------

def rel_block_err(a, b, nblk):
    """max over blocks of ||a_i - b_i||_F / max over blocks ||b_i||_F, per energy, max over energies."""
    a = a.reshape(a.shape[0], nblk, -1)
    b = b.reshape(b.shape[0], nblk, -1)
    num = np.linalg.norm(a - b, axis=2).max(axis=1)
    den = np.maximum(np.linalg.norm(b, axis=2).max(axis=1), 1e-300)
    return float((num / den).max())


def sample_with_peak(ne, k, J):
    """Energies for the FP64 comparison: k evenly spaced over the grid of ne (ends
    included) and the energy where the current J ([ne][interfaces]) is largest in
    magnitude; sorted, without repeats.  Returns (indices, peak index)."""
    J = np.asarray(J).reshape(ne, -1)
    peak = int(np.abs(J).max(axis=1).argmax())
    idx = np.unique(np.append(np.linspace(0, ne - 1, max(1, min(k, ne))).round().astype(int), peak))
    return idx, peak


def current_error(J_mixed, J_ref, grid_max):
    """The scalar reading of the current's error: max over the sampled energies and
    interfaces of |J_mixed - J_ref| / max(|J_ref|, 1e-3 grid_max), with grid_max the
    largest |J| over the whole energy grid."""
    floor = 1e-3 * max(float(grid_max), 1e-300)
    return float((np.abs(J_mixed - J_ref) / np.maximum(np.abs(J_ref), floor)).max())


def observables_vs_fp64(P, ctx, s2, o2, out, idx, w, ne, nb, b):
    """Mixed-vs-FP64 error of the current and the density on the sampled energies.
    The mixed blocks of those energies are gathered into a copy of the FP64 run's
    buffers and both sets go through negf_observables.  J: max over energies and
    interfaces of |dJ| / max(|J64|, 1e-3 max_E |J|) (the scalar reading), with max_E
    over the whole energy grid, taken from the mixed run's current of every energy
    (it agrees with FP64 far below 1e-3 of that maximum; a sample that misses the
    current's peak would otherwise shrink the floor); n: the density summed over the
    sample with the grid's weights, normwise."""
    import torch
    sel = torch.from_numpy(idx).cuda()
    o3 = {kk: (v.clone() if v is not None else None) for kk, v in o2.items()}
    for key, nblk in (("GL_diag", nb), ("GL_low", nb - 1)):
        o3[key].copy_(out[key].view(ne, -1)[sel].reshape(-1))
    ws = w[sel].contiguous()
    res = {}
    for o in (o2, o3):
        P.negf_observables(ctx, s2, o["sigma_L"], ws, o["GR_diag"], o["GR_up"], o["GR_low"], o["GL_diag"],
                           o["GL_low"], None, None, o["current"], o["density"], prec=P.FP64)
    torch.cuda.synchronize()
    J64, Jm = o2["current"].cpu().numpy(), o3["current"].cpu().numpy()
    n64, nm = o2["density"].cpu().numpy(), o3["density"].cpu().numpy()
    J_grid_max = float(out["current"].abs().max().item())
    res["J"] = current_error(Jm, J64, J_grid_max)
    res["n"] = float(np.linalg.norm(nm - n64) / max(np.linalg.norm(n64), 1e-300))
    res["J_max_abs"] = float(np.abs(J64).max())
    res["J_grid_max_abs"] = J_grid_max
    del o3
    return res


def run_gpu(args):
    import torch
    import paper_2602_03438_gb300 as P

    global OZ_SLICE_PAIRS
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ns = P.negf.sliced_digits()
    OZ_SLICE_PAIRS = ns * (ns + 1) / 2.0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    dev = W.config2(nb=args.nb, b=args.b, ne=args.ne)
    dev.energy = rank_energies(args.ne, rank, world)
    prec = {"mixed": P.MIXED, "fp64": P.FP64, "mixed_tf32": P.MIXED_TF32}[args.prec]
    nb, b, ne = dev.nb, dev.b, dev.ne

    ctx = P.Context(local, int(args.workspace_gb * (1 << 30)))
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_)
    fL = torch.from_numpy(dev.f_L()).cuda()
    fR = torch.from_numpy(dev.f_R()).cuda()
    w = torch.from_numpy(rank_weights(args.ne, rank, world)).cuda()
    stream = torch.cuda.current_stream()

    # the OBC products take the sliced FP64-class path with the mixed sweeps, FP64 otherwise
    obc_prec = P.MIXED if prec == P.MIXED else P.FP64

    def obc():
        P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"], prec=obc_prec)

    def rgf(p=prec, s=sys_, o=out, ffL=fL, ffR=fR):
        P.negf_rgf_lesser(ctx, s, p, o["sigma_L"], o["sigma_R"], ffL, ffR, None, o["GR_diag"], o["GR_up"],
                          o["GR_low"], o["GL_diag"], o["GL_low"], o["status"])

    def obs():
        P.negf_observables(ctx, sys_, out["sigma_L"], w, out["GR_diag"], out["GR_up"], out["GR_low"],
                           out["GL_diag"], out["GL_low"], out["T"], out["dos"], out["current"], out["density"],
                           prec=obc_prec)

    def step():
        obc()
        rgf()
        obs()

    for _ in range(args.warmup):
        step()
    if ctx.sync() != 0:
        raise RuntimeError("device status after warm-up")
    bad_obc = int((out["obc_status"] != 0).sum().item())
    bad = int((out["status"] != 0).sum().item())

    # ---- timed region: whole path, K steps, kernel events live
    ctx.profile_reset()
    ctx.profile(True)
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ctx.profile(False)
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world, device=torch.device("cuda", local))
    prof = ctx.profile_read()
    value = world * ne * args.steps / (ms / 1e3)

    # ---- RGF alone (the metric's own definition: Sigma_OBC precomputed)
    barrier(world)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        rgf()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_rgf = max_over_ranks(ev0.elapsed_time(ev1), world, device=torch.device("cuda", local))
    rgf_value = world * ne * args.steps / (ms_rgf / 1e3)

    # ---- FP64 comparison on a bounded subset of the energies (same device, same Sigma)
    cmp = {}
    fp64_sample = 128 if args.fp64_sample is None else args.fp64_sample
    if fp64_sample > 0 and rank == 0:
        # evenly spaced energies and the one where the mixed current peaks, so that the
        # error floor of the current (1e-3 of its largest value over the grid) is itself
        # checked against FP64
        idx, j_peak = sample_with_peak(ne, fp64_sample, out["current"].view(ne, nb - 1).cpu().numpy())
        k = int(idx.size)
        sub = W.config2(nb=args.nb, b=args.b, ne=args.ne)
        sub.energy = dev.energy[idx]
        s2 = P.upload(sub)
        o2 = P.allocate_outputs(s2)
        bb = b * b
        sl = out["sigma_L"].view(ne, bb)[torch.from_numpy(idx).cuda()].reshape(-1)
        sr = out["sigma_R"].view(ne, bb)[torch.from_numpy(idx).cuda()].reshape(-1)
        o2["sigma_L"].copy_(sl)
        o2["sigma_R"].copy_(sr)
        f2L = fL[torch.from_numpy(idx).cuda()].contiguous()
        f2R = fR[torch.from_numpy(idx).cuda()].contiguous()
        rgf(P.FP64, s2, o2, f2L, f2R)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0.record(stream)
        rgf(P.FP64, s2, o2, f2L, f2R)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1)
        fp64_value = k / (ms64 / 1e3)
        # normwise error of each Green's function over its BT pattern, per energy (max over
        # the sampled energies): max block error / max block norm of G^R (diag, up, low)
        # and of G^< (diag, low); the per-family figures are diagnostics
        errs, nums, dens = {}, {}, {}
        for key, nblk in (("GR_diag", nb), ("GR_up", nb - 1), ("GR_low", nb - 1), ("GL_diag", nb),
                          ("GL_low", nb - 1)):
            got = out[key].view(ne, nblk, -1)[torch.from_numpy(idx).cuda()]
            ref = o2[key].view(k, nblk, -1)
            nums[key] = torch.linalg.vector_norm(got - ref, dim=2).amax(dim=1)
            dens[key] = torch.linalg.vector_norm(ref, dim=2).amax(dim=1)
            errs[key] = float((nums[key] / dens[key].clamp_min(1e-300)).max().item())
        joint = {}
        for g, keys in (("G^R", ("GR_diag", "GR_up", "GR_low")), ("G^<", ("GL_diag", "GL_low"))):
            num = torch.stack([nums[x] for x in keys]).amax(0)
            den = torch.stack([dens[x] for x in keys]).amax(0).clamp_min(1e-300)
            joint[g] = float((num / den).max().item())
        obs_err = observables_vs_fp64(P, ctx, s2, o2, out, idx, w, ne, nb, b)
        cmp = {"fp64_rgf_value": fp64_value, "fp64_energies": k, "current_peak_energy_index": j_peak, "speedup_vs_fp64": rgf_value / world / fp64_value,
               "err_vs_fp64_max": max(max(joint.values()), obs_err["J"], obs_err["n"]), "err_vs_fp64": joint,
               "err_observables_vs_fp64": obs_err, "err_per_block_family": errs}
        del o2, s2

    # ---- end to end through host buffers: H2D inputs, the path, D2H observables
    e2e = None
    if not args.no_e2e:
        pin = lambda t: t.cpu().pin_memory()
        h_in = {k: pin(getattr(sys_, k)) for k in ("H_diag", "H_up", "S_diag", "S_up", "energy")}
        h_in.update(fL=pin(fL), fR=pin(fR), w=pin(w))
        d_in = {k: getattr(sys_, k) for k in ("H_diag", "H_up", "S_diag", "S_up", "energy")}
        d_in.update(fL=fL, fR=fR, w=w)
        outs_d2h = ("T", "dos", "current", "density", "status", "obc_status")
        h_out = {k: torch.empty_like(out[k], device="cpu").pin_memory() for k in outs_d2h}
        h2d = sum(t.numel() * t.element_size() for t in h_in.values())
        d2h = sum(t.numel() * t.element_size() for t in h_out.values())
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            for kk, t in h_in.items():
                d_in[kk].copy_(t, non_blocking=True)
            step()
            for kk in outs_d2h:
                h_out[kk].copy_(out[kk], non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms_e2e = max_over_ranks(max(ev0.elapsed_time(ev1), wall * 1e3), world, device=torch.device("cuda", local))
        e2e = {"value": world * ne * args.steps / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": ms_e2e / args.steps,
               "result": "T, DOS, current, density and status arrays"}

    # ---- the energy integrals of the whole grid: every rank's weighted partial sums of
    # the density and the interface currents, summed over the ranks (outside the timed region)
    integrals = energy_integrals(out["density"], out["current"], out["T"], fL, fR, w, ne, nb, world)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peaks, src = measured_peaks()
    cls_ms = {k: v["ms"] for k, v in prof["classes"].items() if v["launches"] > 0}
    dominant = max(cls_ms, key=cls_ms.get)
    roof = roofline_for(dominant, prof["classes"][dominant], peaks, src, sustained=True)
    roof["traffic"] = traffic_for(dominant)
    roof["hbm"] = hbm_for(dominant, peaks, src)
    shares = {k: v / sum(cls_ms.values()) for k, v in cls_ms.items()}

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {P.MIXED: f"bf16 {ns}-digit slices (exact fp32 accumulate) + f32 inverse + f64",
                  P.MIXED_TF32: "tf32x3 + f32 inverse + f64", P.FP64: "f64"}[prec],
        "data": "synthetic",
        "config": {"workload": f"config 2: ballistic batched RGF, nb={nb}, b={b}, {ne} energies/GPU in [-3,3], "
                               "S=I+0.05R, eta=1e-6; step = OBC + G^R/G^< sweeps + observables",
                   "nb": nb, "b": b, "energies_per_gpu": ne, "precision": args.prec,
                   "parallelism": f"energy-sharded x{world}",
                   "l2": "working set larger than L2 (85 GB of G blocks written per step)"},
        "rgf_only": {"value": rgf_value, "unit": UNIT, "ms_per_step": ms_rgf / args.steps},
        "fp64_comparison": cmp,
        "status": {"obc_not_converged": bad_obc, "rgf_flagged": bad},
        "energy_integrals": integrals,
        "gpu_launches": prof["launches"],
        "kernel_time_share": shares,
        "roofline": roof,
        "clocks": clocks,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline(dev, budget_s=args.cpu_budget)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_probe_partitioned(args):
    """Few energies of a long device: --probe partitioned times the sequential G^R sweep
    (negf_rgf_retarded) against the partitioned selected inversion (negf_rgf_partitioned)
    for P = 1, 2, 4, 8, 16 on `ne_cap` energies of the config-2 device lengthened to `nb`
    blocks (default 128), Sigma_OBC precomputed, in the precision of --prec.  Prints one
    JSON line with ms per call and energy points/s per variant and the largest normwise
    G^R difference to the sequential result; not a bench line."""
    import torch
    import paper_2602_03438_gb300 as P
    torch.cuda.set_device(0)
    prec = {"mixed": P.MIXED, "fp64": P.FP64, "mixed_tf32": P.MIXED_TF32}[args.prec]
    nb = args.nb if args.nb != 64 else 128
    full = W.config2(nb=nb, b=args.b, ne=args.ne)
    dev = full.truncated(energies=np.linspace(0, full.ne - 1, args.ne_cap).round().astype(int))
    ctx = P.Context(0, int(args.workspace_gb * (1 << 30)))
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_, lesser=False)
    P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"], prec=P.MIXED)
    ref = {k: torch.empty_like(out[k]) for k in ("GR_diag", "GR_up", "GR_low")}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    seq = lambda: P.negf_rgf_retarded(ctx, sys_, prec, out["sigma_L"], out["sigma_R"], None, ref["GR_diag"],
                                      ref["GR_up"], ref["GR_low"], out["status"])
    res = {"sequential": {"ms_per_call": timed(seq)}}
    for parts in (1, 2, 4, 8, 16):
        if nb % parts or nb // parts < 2:
            continue
        fn = lambda: P.negf_rgf_partitioned(ctx, sys_, prec, parts, out["sigma_L"], out["sigma_R"], None,
                                            out["GR_diag"], out["GR_up"], out["GR_low"], out["status"])
        ms = timed(fn)
        num = max(float(torch.linalg.vector_norm(out[k] - ref[k])) for k in ref)
        den = max(float(torch.linalg.vector_norm(ref[k])) for k in ref)
        res[f"P={parts}"] = {"ms_per_call": ms, "diff_vs_sequential": num / den}
    if ctx.sync() != 0:
        raise RuntimeError("device status after the probe")
    for v in res.values():
        v["energy_points_per_s"] = dev.ne / (v["ms_per_call"] / 1e3)
    print(json.dumps({"probe": "partitioned", "nb": nb, "b": args.b, "energies": dev.ne,
                      "precision": args.prec, "what": "G^R selected blocks, Sigma_OBC precomputed",
                      "results": res}))
    ctx.close()


def run_probe(args):
    """One building block of the sweeps alone, for kernel profiling: --probe gemm runs the
    batched block product D = A B and --probe inverse the block inverse, on `ne` random
    complex128 b x b blocks (config-2 shape by default), `warmup` + `steps` calls, in the
    precision of --prec.  Prints the device time per call; not a bench line."""
    import torch
    import paper_2602_03438_gb300 as P
    torch.cuda.set_device(0)
    prec = {"mixed": P.MIXED, "fp64": P.FP64, "mixed_tf32": P.MIXED_TF32}[args.prec]
    gen = torch.Generator(device="cuda").manual_seed(20260002)
    shape = (args.ne, args.b, args.b)
    A = torch.randn(shape, dtype=torch.complex128, device="cuda", generator=gen)
    B = torch.randn(shape, dtype=torch.complex128, device="cuda", generator=gen)
    if args.probe == "inverse":   # diagonally dominant: well conditioned blocks
        A = A + args.b * torch.eye(args.b, dtype=torch.complex128, device="cuda")
    D = torch.empty_like(A)
    ctx = P.Context(0, int(args.workspace_gb * (1 << 30)))
    call = (lambda: P.negf.negf_block_gemm(ctx, prec, A, B, D)) if args.probe == "gemm" else \
        (lambda: P.negf.negf_block_inverse(ctx, prec, A, D))
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        call()
    e1.record()
    torch.cuda.synchronize()
    if ctx.sync() != 0:
        raise RuntimeError("device status after the probe")
    print(json.dumps({"probe": args.probe, "b": args.b, "units": args.ne, "precision": args.prec,
                      "ms_per_call": e0.elapsed_time(e1) / args.steps}))
    ctx.close()


def run_config4(args):
    """Config 4 at its stated size: nb = 32, b = 512, all 512 energies, block-diagonal
    scattering.  The Green's function blocks of all energies would take 343 GB, so the
    sweeps and observables run chunk by chunk in the workspace (negf_rgf_observables):
    one timed run of OBC + sweeps + T, DOS, current and density over every energy, mixed
    precision; then the current of `fp64_sample` sampled energies from the FP64 sweeps
    (blocks stored, same Sigma) against the mixed run's (|dJ| / max(|J|, 1e-3 max|J|))."""
    import torch
    import paper_2602_03438_gb300 as P
    torch.cuda.set_device(0)
    dev = W.config4()
    ctx = P.Context(0, int(args.workspace_gb * (1 << 30)))
    sys_ = P.upload(dev)
    L = sys_.layout()[-1]
    cz = lambda n: torch.empty(int(n), dtype=torch.complex128, device="cuda")
    z64 = lambda n: torch.zeros(int(n), dtype=torch.float64, device="cuda")
    sig_L, sig_R = cz(L[3]), cz(L[3])
    st_obc = torch.zeros(dev.ne, dtype=torch.int32, device="cuda")
    status = torch.zeros(dev.ne, dtype=torch.int32, device="cuda")
    iters = torch.zeros(2 * dev.ne, dtype=torch.int32, device="cuda")
    T, dos, J, n = z64(L[2]), z64(L[2]), z64(L[6]), z64(L[7])
    fL = torch.from_numpy(dev.f_L()).cuda()
    fR = torch.from_numpy(dev.f_R()).cuda()
    w = torch.from_numpy(dev.weights()).cuda()
    sc = P.Scattering.from_devices([dev])
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    P.negf_obc(ctx, sys_, sig_L, sig_R, iters, st_obc, prec=P.MIXED)
    e1.record()
    P.negf.negf_rgf_observables(ctx, sys_, P.MIXED, sig_L, sig_R, fL, fR, sc, w, T, dos, J, n, status)
    e2.record()
    torch.cuda.synchronize()
    if ctx.sync() != 0:
        raise RuntimeError("device status after the config-4 run")
    ms_obc, ms_sw = e0.elapsed_time(e1), e1.elapsed_time(e2)
    # FP64 sweeps with stored blocks on sampled energies, same Sigma: evenly spaced ones
    # and the energy where the mixed current peaks (so that the current is checked where
    # it is largest, not only against the floor of 1e-3 of the grid's largest current)
    J_all = J.cpu().numpy().reshape(dev.ne, dev.nb - 1)
    idx, j_peak = sample_with_peak(dev.ne, 4 if args.fp64_sample is None else args.fp64_sample, J_all)
    k = len(idx)
    sub = dev.truncated(energies=idx)
    s2 = P.upload(sub)
    o2 = P.allocate_outputs(s2)
    sel = torch.from_numpy(idx).cuda()
    bb = dev.b * dev.b
    o2["sigma_L"].copy_(sig_L.view(dev.ne, bb)[sel].reshape(-1))
    o2["sigma_R"].copy_(sig_R.view(dev.ne, bb)[sel].reshape(-1))
    sc2 = P.Scattering.from_devices([sub])
    f2L, f2R = fL[sel].contiguous(), fR[sel].contiguous()
    P.negf_rgf_lesser(ctx, s2, P.FP64, o2["sigma_L"], o2["sigma_R"], f2L, f2R, sc2, o2["GR_diag"], o2["GR_up"],
                      o2["GR_low"], o2["GL_diag"], o2["GL_low"], o2["status"])
    P.negf_observables(ctx, s2, o2["sigma_L"], None, None, None, None, None, o2["GL_low"], None, None,
                       o2["current"], None, prec=P.FP64)
    torch.cuda.synchronize()
    J64 = o2["current"].cpu().numpy().reshape(k, dev.nb - 1)
    Jm = J_all[idx]
    J_grid_max = float(np.abs(J_all).max())   # max_E over all energies (mixed)
    line = {"workload": "config4", "devices": 1, "energies": dev.ne, "nb": dev.nb, "b": dev.b,
            "mixed": {"value": dev.ne / ((ms_obc + ms_sw) / 1e3), "unit": UNIT, "ms_per_run": ms_obc + ms_sw,
                      "ms_obc": ms_obc, "ms_sweeps_and_observables": ms_sw,
                      "what": "OBC + G^R/G^< sweeps + T, DOS, current, density over all 512 energies, mixed "
                              "precision, blocks kept in the workspace chunk by chunk (negf_rgf_observables)"},
            "J_err_vs_fp64": current_error(Jm, J64, J_grid_max),
            "J_err_at_peak_vs_fp64": float(np.abs(Jm[list(idx).index(j_peak)] - J64[list(idx).index(j_peak)]).max() /
                                           np.abs(J64[list(idx).index(j_peak)]).max()),
            "fp64_sampled_energies": idx.tolist(), "current_peak_energy_index": j_peak,
            "finite": bool(np.isfinite(J.cpu().numpy()).all() and np.isfinite(n.cpu().numpy()).all()),
            "status": {"obc_not_converged": int((st_obc != 0).sum().item()),
                       "rgf_flagged": int((status != 0).sum().item())}}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_config1(args):
    """Config 1, the small latency-bound case (nb 16, b 8, 64 energies): microseconds per
    batch of all 64 energies for OBC + G^R/G^< sweeps + observables, per precision (b = 8
    is below the sliced product's smallest block, so NEGF_MIXED takes the FP64 products
    here and differs from NEGF_FP64 only in its FP32 inverses with refinement), and the
    largest normwise G^R difference between the two precisions (the parity tests compare
    config 1 with the CPU oracle).  Not a bench line."""
    import torch
    import paper_2602_03438_gb300 as P
    torch.cuda.set_device(0)
    dev = W.config1()
    ctx = P.Context(0, 256 << 20)
    sys_ = P.upload(dev)
    out = P.allocate_outputs(sys_)
    fL = torch.from_numpy(dev.f_L()).cuda()
    fR = torch.from_numpy(dev.f_R()).cuda()
    w = torch.from_numpy(dev.weights()).cuda()
    res = {}
    GR64 = None
    for name, prec in (("fp64", P.FP64), ("mixed", P.MIXED)):
        def step():
            P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"], prec=prec)
            P.negf_rgf_lesser(ctx, sys_, prec, out["sigma_L"], out["sigma_R"], fL, fR, None, out["GR_diag"],
                              out["GR_up"], out["GR_low"], out["GL_diag"], out["GL_low"], out["status"])
            P.negf_observables(ctx, sys_, out["sigma_L"], w, out["GR_diag"], out["GR_up"], out["GR_low"],
                               out["GL_diag"], out["GL_low"], out["T"], out["dos"], out["current"],
                               out["density"], prec=prec)
        for _ in range(max(args.warmup, 1)):
            step()
        if ctx.sync() != 0:
            raise RuntimeError("device status after the warm-up")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(max(args.steps, 1)):
            e0.record()
            step()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) * 1e3)
        GR = out["GR_diag"].cpu().numpy().reshape(dev.ne, -1)
        res[name] = {"us_per_batch_median": float(np.median(times)), "us_per_batch_min": float(np.min(times))}
        if GR64 is None:
            GR64 = GR
        else:
            res[name]["GR_err_vs_fp64"] = float((np.linalg.norm(GR - GR64, axis=1) /
                                                 np.linalg.norm(GR64, axis=1)).max())
    # the sweeps and observables (mixed) as one CUDA graph captured on the caller's stream
    # (they make no host synchronisation; the OBC polls the host between its steps and
    # stays outside, its Sigma from the last run): the launch overhead of the small case
    def sweeps_obs():
        P.negf_rgf_lesser(ctx, sys_, P.MIXED, out["sigma_L"], out["sigma_R"], fL, fR, None, out["GR_diag"],
                          out["GR_up"], out["GR_low"], out["GL_diag"], out["GL_low"], out["status"])
        P.negf_observables(ctx, sys_, out["sigma_L"], w, out["GR_diag"], out["GR_up"], out["GR_low"],
                           out["GL_diag"], out["GL_low"], out["T"], out["dos"], out["current"], out["density"],
                           prec=P.MIXED)
    try:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            sweeps_obs()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        direct = {k: out[k].clone() for k in ("GR_diag", "GL_diag", "current", "density")}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_direct = []
        for _ in range(max(args.steps, 1)):
            e0.record()
            sweeps_obs()
            e1.record()
            torch.cuda.synchronize()
            t_direct.append(e0.elapsed_time(e1) * 1e3)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            sweeps_obs()
        t_graph = []
        for _ in range(max(args.steps, 1)):
            e0.record()
            graph.replay()
            e1.record()
            torch.cuda.synchronize()
            t_graph.append(e0.elapsed_time(e1) * 1e3)
        same = all(bool(torch.equal(direct[k], out[k])) for k in direct)
        res["sweeps_and_observables_mixed"] = {"us_per_batch_direct": float(np.median(t_direct)),
                                               "us_per_batch_graph": float(np.median(t_graph)),
                                               "graph_replay_bit_identical": same}
    except Exception as ex:   # a capture the runtime refuses is reported, not fatal
        res["sweeps_and_observables_mixed"] = {"graph_error": str(ex)[:300]}
    print(json.dumps({"workload": "config1", "nb": dev.nb, "b": dev.b, "energies": dev.ne,
                      "what": "OBC + G^R/G^< sweeps + T, DOS, current, density for all 64 energies, one batch",
                      **res}), flush=True)


def run_workload(args):
    """Mixed vs FP64 on the other workloads (not the headline line): --workload config4 runs
    the nb = 32, b = 512 device with block-diagonal scattering over `ne` energies;
    --workload config3 runs the first `devices` devices of the uneven batch (every energy).
    Times OBC + G^R/G^< sweeps in mixed precision over the whole set, then the FP64 sweeps
    on a sample of `fp64_sample` energies per device with the same Sigma, and reports the
    normwise error of the mixed G^R, G^< against FP64 over the BT pattern."""
    import torch
    import paper_2602_03438_gb300 as P
    torch.cuda.set_device(0)
    # the outputs stay resident: config 4 keeps 628 MB of blocks per energy, config 3's
    # largest devices 640 MB, so the energies are capped to fit the GPU's memory
    if args.workload == "config4":
        full = W.config4()
        devs = [full.truncated(energies=np.linspace(0, full.ne - 1, args.ne_cap).round().astype(int))]
    else:
        shapes = W.config3_shapes()
        devs = []
        for k in range(args.devices):
            d = W.config3_device(k, shapes)
            devs.append(d.truncated(energies=np.linspace(0, d.ne - 1, min(args.ne_cap, d.ne)).round().astype(int)))
    ctx = P.Context(0, int(args.workspace_gb * (1 << 30)))
    # tile shapes of the block products: the autotuner's choice per block size
    tuned = P.tuning.tune(ctx, sorted(set(d.b for d in devs)), units=256)["choices"]
    sys_ = P.upload(devs)
    out = P.allocate_outputs(sys_)
    sc = P.Scattering.from_devices(devs) if devs[0].sigR_scat is not None else None
    fL = torch.from_numpy(np.concatenate([d.f_L() for d in devs])).cuda()
    fR = torch.from_numpy(np.concatenate([d.f_R() for d in devs])).cuda()
    ne_tot = sum(d.ne for d in devs)

    def step():
        P.negf_obc(ctx, sys_, out["sigma_L"], out["sigma_R"], out["iters"], out["obc_status"], prec=P.MIXED)
        P.negf_rgf_lesser(ctx, sys_, P.MIXED, out["sigma_L"], out["sigma_R"], fL, fR, sc, out["GR_diag"],
                          out["GR_up"], out["GR_low"], out["GL_diag"], out["GL_low"], out["status"])

    def sweeps():
        P.negf_rgf_lesser(ctx, sys_, P.MIXED, out["sigma_L"], out["sigma_R"], fL, fR, sc, out["GR_diag"],
                          out["GR_up"], out["GR_low"], out["GL_diag"], out["GL_low"], out["status"])

    step()
    if ctx.sync() != 0:
        raise RuntimeError("device status after the first run")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the sweeps alone (Sigma_OBC precomputed), with the kernel launch count
    ctx.profile_reset()
    e0.record()
    for _ in range(args.steps):
        sweeps()
    e1.record()
    torch.cuda.synchronize()
    ms_sw = e0.elapsed_time(e1) / args.steps
    launches_sw = ctx.profile_read()["launches"] / args.steps
    # FP64 sweeps on a sample of each device's energies, given the mixed run's Sigma
    L = sys_.layout()
    subs, idx_all = [], []
    for d, dev in enumerate(devs):
        k = min(1 if args.fp64_sample is None else args.fp64_sample, dev.ne)
        idx = np.linspace(0, dev.ne - 1, k).round().astype(int)
        subs.append(dev.truncated(energies=idx))
        idx_all.append((d, idx))
    s2 = P.upload(subs)
    o2 = P.allocate_outputs(s2)
    L2 = s2.layout()
    for (d, idx), sub in zip(idx_all, subs):
        b = sub.b
        for j, e in enumerate(idx):
            src = slice(int(L[d][3] + e * b * b), int(L[d][3] + (e + 1) * b * b))
            dst = slice(int(L2[d][3] + j * b * b), int(L2[d][3] + (j + 1) * b * b))
            o2["sigma_L"][dst] = out["sigma_L"][src]
            o2["sigma_R"][dst] = out["sigma_R"][src]
    sc2 = P.Scattering.from_devices(subs) if subs[0].sigR_scat is not None else None
    f2L = torch.from_numpy(np.concatenate([d.f_L() for d in subs])).cuda()
    f2R = torch.from_numpy(np.concatenate([d.f_R() for d in subs])).cuda()
    torch.cuda.synchronize()
    e0.record()
    P.negf_rgf_lesser(ctx, s2, P.FP64, o2["sigma_L"], o2["sigma_R"], f2L, f2R, sc2, o2["GR_diag"], o2["GR_up"],
                      o2["GR_low"], o2["GL_diag"], o2["GL_low"], o2["status"])
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    n64 = sum(len(i) for _, i in idx_all)
    err = {"G^R": 0.0, "G^<": 0.0}
    for (d, idx), sub in zip(idx_all, subs):
        nb, b = sub.nb, sub.b
        for gname, keys in (("G^R", (("GR_diag", nb), ("GR_up", nb - 1), ("GR_low", nb - 1))),
                            ("G^<", (("GL_diag", nb), ("GL_low", nb - 1)))):
            for j, e in enumerate(idx):
                num = den = 0.0
                for key, nblk in keys:
                    if nblk == 0:
                        continue
                    off = 4 if key.endswith("diag") else 5
                    a0 = int(L[d][off] + e * nblk * b * b)
                    b0 = int(L2[d][off] + j * nblk * b * b)
                    got = out[key][a0:a0 + nblk * b * b].view(nblk, -1)
                    ref = o2[key][b0:b0 + nblk * b * b].view(nblk, -1)
                    num = max(num, float(torch.linalg.vector_norm(got - ref, dim=1).max()))
                    den = max(den, float(torch.linalg.vector_norm(ref, dim=1).max()))
                err[gname] = max(err[gname], num / max(den, 1e-300))
    line = {"workload": args.workload, "devices": len(devs), "energies": ne_tot,
            "block_sizes": sorted(set(d.b for d in devs)),
            "mixed": {"value": ne_tot / (ms / 1e3), "unit": UNIT, "ms_per_run": ms,
                      "what": "OBC + G^R/G^< sweeps, mixed precision, every energy"},
            "mixed_sweeps": {"value": ne_tot / (ms_sw / 1e3), "unit": UNIT, "ms_per_run": ms_sw,
                             "launches_per_run": launches_sw,
                             "what": "G^R/G^< sweeps alone (Sigma_OBC precomputed): devices of one block "
                                     "size sweep together, one launch per step over all their units"},
            "fp64_sweeps": {"value": n64 / (ms64 / 1e3), "unit": UNIT, "energies": n64},
            "err_vs_fp64": err,
            "tuned_variants": {n: v["variant"] for n, v in tuned.items()},
            "status": {"obc_not_converged": int((out["obc_status"] != 0).sum().item()),
                       "rgf_flagged": int((out["status"] != 0).sum().item())}}
    print(json.dumps(line), flush=True)
    ctx.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64", "mixed_tf32"])
    ap.add_argument("--nb", type=int, default=64)
    ap.add_argument("--b", type=int, default=128)
    ap.add_argument("--ne", type=int, default=1024)
    ap.add_argument("--workspace-gb", type=float, default=24.0)
    ap.add_argument("--fp64-sample", type=int, default=None,
                    help="energies per device of the FP64 comparison (default: 128 for the bench line, "
                         "4 for --workload config4, 1 for --workload config3)")
    ap.add_argument("--ref-energies", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--probe", choices=["gemm", "inverse", "partitioned"], default=None)
    ap.add_argument("--workload", choices=["config1", "config3", "config4"], default=None)
    ap.add_argument("--devices", type=int, default=16)
    ap.add_argument("--ne-cap", type=int, default=64)
    args = ap.parse_args(argv)
    if args.probe == "partitioned":
        run_probe_partitioned(args)
    elif args.probe:
        run_probe(args)
    elif args.workload == "config4":
        run_config4(args)
    elif args.workload == "config1":
        run_config1(args)
    elif args.workload:
        run_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
