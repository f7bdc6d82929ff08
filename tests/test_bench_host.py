"""Host logic of bench.py on CPU: energy sharding across ranks, the
max-over-ranks timing reduction (2 gloo ranks), clock parsing, roofline math."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def test_rank_energies_partition_the_grid():
    ne, world = 1024, 4
    parts = [bench.rank_energies(ne, r, world) for r in range(world)]
    assert all(p.size == ne for p in parts)
    allv = np.sort(np.concatenate(parts))
    assert np.array_equal(allv, np.linspace(-3.0, 3.0, ne * world))
    # interleaved: every rank spans the whole window
    assert all(p.min() < -2.9 and p.max() > 2.9 for p in parts)
    # one rank is exactly the single-GPU workload
    assert np.array_equal(bench.rank_energies(ne, 0, 1), np.linspace(-3.0, 3.0, ne))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.max_over_ranks(10.0 + rank, world)
    e = bench.rank_energies(8, rank, world)
    bench.barrier(world)
    q.put((rank, v, e.tolist()))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]
    e0, e1 = res[0][2], res[1][2]
    assert not set(e0) & set(e1) and len(e0) == len(e1) == 8


def test_clock_summary_parsing():
    c = bench.ClockSampler(0)
    c.lines = ["0, 1900, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1800, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2000, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["sm_mhz"] == 1900.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_roofline_arithmetic():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1650.0}
    st = {"launches": 10, "ms": 20.0, "flops": 10 * 8 * 128 ** 3 * 1024.0, "bytes": 0.0}
    r = bench.roofline_for("gemm_tc", st, peaks, "measured")
    per = 8 * 128 ** 3 * 1024.0 / 2e-3 / 1e12
    assert abs(r["achieved"] - per) < 1e-9
    assert abs(r["peak"] - 1650.0 * 1.1 / 2.25 / 3) < 1e-9
    assert abs(r["frac"] - per / r["peak"]) < 1e-12
    r2 = bench.roofline_for("gemm_f64", st, peaks, "measured")
    assert r2["bound"] == "alu" and r2["peak"] == 1.25


def test_roofline_sliced_gemm_counts_useful_work_against_tf32_third():
    """The sliced product's roofline counts the useful 8 n^3 flops of a complex product
    against the useful peak of a complex product on the tensor cores (TF32 peak / 3,
    TF32 = bf16 x 1.1/2.25); the executed BF16 work (OZ_SLICE_PAIRS slice pairs per
    complex product) is reported beside."""
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1650.0}
    st = {"launches": 4, "ms": 8.0, "flops": 4 * 8 * 128 ** 3 * 100.0, "bytes": 0.0}
    r = bench.roofline_for("gemm_oz", st, peaks, "measured")
    useful = 8 * 128 ** 3 * 100.0 / 2e-3 / 1e12
    assert abs(r["useful_tflops"] - useful) < 1e-9
    assert abs(r["achieved"] - useful) < 1e-9
    assert abs(r["peak"] - 1650.0 * 1.1 / 2.25 / 3.0) < 1e-9
    assert abs(r["frac"] - useful / r["peak"]) < 1e-12
    pairs = bench.OZ_SLICE_PAIRS
    assert pairs == 36.0   # 8 digits, s + t <= 9 (the library default)
    assert abs(r["executed_bf16_tflops"] - pairs * useful) < 1e-9
    assert abs(r["executed_bf16_frac"] - pairs * useful / 1650.0) < 1e-12


def test_traffic_record_matches_the_kernel_source(tmp_path, monkeypatch):
    """The committed per-product DRAM traffic is reported only while the kernel source
    it was captured from is unchanged (its hash recorded beside the figure)."""
    import hashlib
    import json
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "roofline_traffic.json")))["gemm_oz"]
    src = os.path.join(bench.ROOT, rec["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    expect = rec["bytes_per_launch_full"] if h == rec["source_sha256_16"] else None
    assert bench.traffic_for("gemm_oz") == expect
    # at least the algorithmic bytes of one product (A, B read and D written once)
    assert rec["bytes_per_launch_full"] >= 3 * 1024 * 128 * 128 * 16
    # a changed source makes the figure stale: null
    fake = tmp_path / "profiles"
    fake.mkdir()
    (tmp_path / "k.cu").write_text("changed")
    (fake / "roofline_traffic.json").write_text(json.dumps(
        {"gemm_oz": {"source": "k.cu", "source_sha256_16": h, "bytes_per_launch_full": 1}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("gemm_oz") is None
    assert bench.traffic_for("inv_f32") is None


def _integral_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ne, nb, norb = 16, 5, 3
    E = bench.rank_energies(ne, rank, world)
    w = torch.from_numpy(bench.rank_weights(ne, rank, world))
    # a rank's outputs as negf_observables leaves them: its weighted density sum, the
    # per-energy interface currents (conserved: T (f_L - f_R) at every interface)
    nE = np.stack([np.cos(E * (k + 1)) for k in range(norb)], axis=1)            # [ne][orbitals]
    density = torch.from_numpy((w.numpy()[:, None] * nE).sum(0))
    T = torch.from_numpy(np.exp(-E * E))
    fL = torch.from_numpy(1.0 / (1.0 + np.exp((E - 0.5) / 0.3)))
    fR = torch.from_numpy(1.0 / (1.0 + np.exp((E + 0.5) / 0.3)))
    J = (T * (fL - fR)).numpy()
    current = torch.from_numpy(np.repeat(J[:, None], nb - 1, axis=1).reshape(-1).copy())
    out = bench.energy_integrals(density, current, T, fL, fR, w, ne, nb, world)
    q.put((rank, out))
    dist.destroy_process_group()


def test_energy_integrals_sum_over_two_gloo_ranks():
    """The ranks' weighted partial sums add up to the trapezoid integral over the whole
    grid (the exchange step of energy-sharded runs)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_integral_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=120) for _ in ps), key=lambda x: x[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    grid = np.linspace(-3.0, 3.0, 32)
    dens_ref = sum(np.trapezoid(np.cos(grid * (k + 1)), grid) for k in range(3))
    f = lambda mu: 1.0 / (1.0 + np.exp((grid - mu) / 0.3))
    cur_ref = np.trapezoid(np.exp(-grid * grid) * (f(0.5) - f(-0.5)), grid)
    for _, out in res:
        assert out["collective"] == "all_reduce sum over 2 ranks"
        assert abs(out["density_total"] - dens_ref) < 1e-12
        for k in ("current_interface_first", "current_interface_last", "current_landauer"):
            assert abs(out[k] - cur_ref) < 1e-12


def test_rank_weights_one_rank_is_the_local_trapezoid():
    assert np.array_equal(bench.rank_weights(64, 0, 1), bench.W.trapezoid_weights(np.linspace(-3.0, 3.0, 64)))
    parts = [bench.rank_weights(8, r, 4) for r in range(4)]
    assert abs(sum(p.sum() for p in parts) - 6.0) < 1e-12


def test_current_error_floor_comes_from_the_whole_grid():
    """The scalar reading |dJ| / max(|J|, 1e-3 max_E |J|) with max_E over the whole
    energy grid: a tiny current far below the grid's peak is measured against the floor,
    an energy above the floor against its own value."""
    J_ref = np.array([[1e-9, 2e-9], [5e-4, 5e-4]])
    J_mix = J_ref + np.array([[1e-12, -1e-12], [5e-10, 0.0]])
    # grid peak 3e-3: floor 3e-6, so the tiny entries count 1e-12 / 3e-6
    assert abs(bench.current_error(J_mix, J_ref, 3e-3) - 1e-6) < 1e-15
    # a floor from the sample alone (peak 5e-4 -> 5e-7) would count them 2e-6
    assert abs(bench.current_error(J_mix, J_ref, 5e-4) - 2e-6) < 1e-15
    assert bench.current_error(J_ref, J_ref, 3e-3) == 0.0


def test_hbm_bandwidth_from_the_traffic_record():
    rec = bench.traffic_record("gemm_oz")
    if rec is None:
        pytest.skip("the record does not match the current kernel source")
    peaks = {"hbm_gbs": 6000.0}
    h = bench.hbm_for("gemm_oz", peaks, "test")
    gbs = rec["bytes_per_launch_full"] / (rec["ms_per_launch_full"] / 1e3) / 1e9
    assert abs(h["achieved_gbs"] - gbs) < 1e-9 * gbs and abs(h["frac"] - gbs / 6000.0) < 1e-12


def test_fp64_sample_includes_the_current_peak():
    """The FP64 comparison's energies: evenly spaced, ends included, plus the energy of
    the largest current (once, in order), which a sparse sample would otherwise miss."""
    ne = 512
    J = np.zeros((ne, 31))
    J[261, 7] = -3e-3        # the peak, by magnitude and negative
    J[10, 0] = 1e-3
    idx, peak = bench.sample_with_peak(ne, 4, J)
    assert peak == 261
    assert idx.tolist() == [0, 170, 261, 341, 511]
    # a peak that is already a sample point is not repeated
    J2 = np.zeros((ne, 3))
    J2[341, 1] = 1.0
    idx2, peak2 = bench.sample_with_peak(ne, 4, J2)
    assert peak2 == 341 and idx2.tolist() == [0, 170, 341, 511]
    # k above ne: every energy once
    idx3, _ = bench.sample_with_peak(5, 128, np.arange(10.0).reshape(5, 2))
    assert idx3.tolist() == [0, 1, 2, 3, 4]
