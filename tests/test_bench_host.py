"""Host logic of bench.py: the cross-rank reduction of the N > 1 (replica) path
runs over gloo with two CPU ranks; the efficiency metric of Sec. 4.1.3."""
import math
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    q.put((rank, bench.max_over_ranks(1.5 + rank, dist)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 2.5, 1: 2.5}


def test_single_process_and_efficiency():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert math.isclose(bench.efficiency(1.0, 1e-8, 100), 0.08)


def test_roofline_picks_dominant_kernel_and_scales_traffic():
    """The roofline object: algorithmic flops of the units over the summed event
    time, against the FP32 / double-float peaks derived from the device's SM
    count and the sampled clock; the kernel with the larger total time is
    reported and the other attached; the DRAM traffic of a launch scales with
    the units it processed."""
    import bench
    geom = (48, 48, 48, 288, 20)
    peaks = {"hbm_gbs": 6800.0}
    dev = {"sms": 152, "fp32_fma_tflops": 78.0, "fp64_fma_tflops": 1.2, "fp32_butterfly_tflops": 60.0,
           "df64_butterfly_tflops": 6.5, "sm_clock_mhz": 2070.0}
    alu = bench.alu_peaks(dev, 2070.0)
    assert math.isclose(alu["fp32"], 152 * 128 * 2 * 2.07e9 / 1e12)
    assert math.isclose(alu["df64"], alu["fp32"] / 2 / bench.DF64_INSTR_PER_FLOP)
    d = dict(ms_fp32=20.0, units_fp32=40000, calls_fp32=300, ms_fp64=25.0, units_fp64=7000, calls_fp64=35)
    r = bench.roofline(d, geom, peaks, alu, dev)
    assert r["kernel"].startswith("k_plane_sw<48,48>")                   # 25 ms > 20 ms
    _, f64 = bench.plane_pass_work(geom, 8)
    assert math.isclose(r["achieved"], 7000 * f64 / 25e-3 / 1e12, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / alu["df64"], rel_tol=1e-12)
    assert math.isclose(r["traffic"], bench.TRAFFIC_PER_UNIT["k_plane_sw"] * 7000 / 35, rel_tol=1e-12)
    o = r["other_plane_kernel"]
    _, f32 = bench.plane_pass_work(geom, 4)
    assert math.isclose(o["frac"], 40000 * f32 / 20e-3 / 1e12 / alu["fp32"], rel_tol=1e-12)
    # another grid: no traffic figure (the captures are of the 48^3 grid)
    assert bench.roofline(d, (32, 32, 32, 200, 15), peaks, alu, dev)["traffic"] is None
    assert bench.roofline(dict(d, ms_fp64=0.0, units_fp64=0), geom, peaks, alu, dev)["kernel"].startswith("k_plane_rc")
    r0 = bench.roofline(d, geom, peaks, alu, dev, fp32_kernel="k_plane_r", df64_kernel="k_plane_t")
    assert r0["kernel"].startswith("k_plane_t<dfloat") and r0["other_plane_kernel"]["kernel"].startswith("k_plane_r<")
