"""The multi-rank path of bench.py on CPU.  The method's units are independent,
so N GPUs run N replicas with no collective on the data path; the only
cross-rank steps are the barriers around the timed region and the maximum of
the ranks' times.  Two gloo ranks check that step and the job throughput; the
reference arm returns at once on every rank but 0."""
import argparse
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, ms_by_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = bench.max_over_ranks(ms_by_rank[rank], dist, "cpu")
    out.put((rank, ms, bench.job_throughput(world, 10, 505, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, [10.0, 12.5], out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in got:
        assert ms == 12.5
        assert value == pytest.approx(2 * 10 * 505 / 12.5e-3)


def test_single_process_keeps_its_own_time():
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
    assert bench.job_throughput(1, 4, 100, 8.0) == pytest.approx(4 * 100 / 8e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(workload="mixed_ecc", steps=1, warmup=0, gpus=2, refine=None)
    assert bench.run_reference(args) == 0


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` on the host cores: one JSON line with the
    contract's keys, the oracle as the reference, no host-device bytes."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                        "fp64_small", "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_host_core_samples_run_on_a_small_case():
    """The bench's host-core samples (the oracle's piCholesky and exact CV, and
    NumPy's LAPACK exact CV) return positive rates with their descriptions."""
    from paper_1404_0466_gb300 import synth
    prob = synth.fp64_small(n=512, d=64)
    cfg = dict(synth.FP64_SMALL, n=512, d=64)
    for fn in (bench.oracle_exact_sample, bench.lapack_sample):
        out = fn(prob, cfg)
        assert out["value"] > 0 and out["unit"] == "evals/s" and out["cores"] >= 1 and out["sample"]


def test_roofline_entry_arithmetic():
    """achieved = algorithmic work per launch / average launch time, frac =
    achieved / peak; the work is the method's (each product counted once), the
    kernel's extra arithmetic is a separate factor, and an ALU-bound stage is
    measured against the probed FP32 rate when the bench has it."""
    from paper_1404_0466_gb300 import synth
    cfg = dict(synth.MIXED_ECC)
    work = bench.stage_work(cfg, "mixed", 1, residual="double_float")
    kind, amount, bound, executed = work["resid"]
    assert kind == "flop" and bound == "alu" and executed > 5
    tkind, tamount, tbound, texec = bench.stage_work(cfg, "mixed", 1)["resid"]
    assert tbound == "tensor" and tamount == amount and texec > 9
    # one residual per (fold, lambda): 2 d^2 c for the two triangular products and
    # 2 (r+1) D for one evaluation of the factor; 505 pairs of the mixed case
    d, c, p = 2048, 10, 4
    D = d * (d + 1) // 2
    assert amount == 5 * 101 * (2 * d * d * c + 2 * p * D)
    assert abs(amount - 50.84e9) < 0.01e9
    kind, amount_g, bound, executed = work["gram"]
    assert amount_g == 32768 * d * (d + 1) and bound == "tensor" and executed == 3
    # the trailing updates run on the CUDA cores unless the tuning picks the tensor cores
    assert work["chol_update"][2:] == ("alu", 1)
    assert bench.stage_work(cfg, "mixed", 1, update_engine=0)["chol_update"][2:] == ("tensor", 3)
    # the direct-form score computes Y_f - X_f W: 3 products of 2 (n / k) d c per system
    # against the 2 d^2 c of <W, G_f W>
    kind, amount_s, bound, executed = work["score"]
    assert amount_s == 5 * 101 * 2 * d * d * c and bound == "tensor"
    assert abs(executed - 3 * 32768 / (5 * d)) < 1e-12
    peaks = {"hbm_gbs": 6695.0, "pipes": {"fp32_fma_tflops": 77.0, "fp64_fma_tflops": 1.06}}
    info = bench.roofline_of("resid", 9.0, 30, cfg, "mixed", 1, 10, peaks, work=work)
    per_launch = amount / 3.0
    assert abs(info["work_per_launch"] - per_launch) < 1e-6 * per_launch
    assert abs(info["achieved"] - per_launch / (9.0e-3 / 30) / 1e12) < 1e-9 * info["achieved"]
    assert info["peak"] == 77.0
    assert abs(info["frac"] - info["achieved"] / info["peak"]) < 1e-12
    assert abs(info["issue_rate"] - info["achieved"] * info["executed_per_algorithmic"]) < 1e-9
    top = bench.roofline({"resid": (9.0, 30), "solve": (5.0, 20)}, cfg, "mixed", 1, 10, peaks,
                         work=work, workload="mixed_ecc")
    assert top["kernel_stage"] == "resid" and top["traffic"] is None
    assert bench.roofline_of("chol_diag", 1.0, 32, cfg, "mixed", 1, 1, peaks, work=work)["peak"] == 1.06
    # without a probe the derived FP32 figure stands in
    assert bench.roofline_of("resid", 9.0, 30, cfg, "mixed", 1, 10, {}, work=work)["peak"] == bench.FP32_PEAK_TFLOPS


def test_clock_samples_are_summarised():
    ok = "0, 2070 MHz, 2070 MHz, 1010.52 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1965 MHz, 2070 MHz, 1398.02 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500 MHz, 2070 MHz, 1200.00 W, 0x0000000000000008, Active, Not Active, Not Active, Not Active"
    got = bench.summarise_clocks([ok, ok, capped, "", "garbage", "0, [N/A], 2070 MHz, 1 W, 0x0, a, b, c, d"])
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    got = bench.summarise_clocks([ok, hot, capped])
    assert got["sm_mhz"] == 1965.0 and got["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.summarise_clocks([])["reasons"] == ["no samples"]
