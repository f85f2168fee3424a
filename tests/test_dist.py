"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the job
time is the slowest rank's, and the value counts the walker-steps of every
rank (the sharded population itself: tests/test_sharded.py)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    t = bench.max_over_ranks(100.0 + 50.0 * rank)
    out.put((r, ws, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_seeds():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[2] == 150.0 for x in res)  # the slowest rank's time on both


def test_job_throughput_counts_all_ranks():
    import bench

    assert bench.job_throughput(512, 10, 1000.0, 1) == 5120.0
    assert bench.job_throughput(512, 10, 1000.0, 4) == 4 * 5120.0
    assert bench.max_over_ranks(7.5) == 7.5  # no process group: local value


def test_l2_note_states_whether_the_inputs_fit_in_l2():
    """The bench line says whether a step's inputs exceed the 129 MB L2 (no
    flush between steps is needed then) or are L2-resident."""
    import bench
    import workloads

    assert bench.l2_note(workloads.config("c2")).startswith("inputs larger than L2 (packed L 650 MB")
    for c in ("c0", "c1"):
        assert bench.l2_note(workloads.config(c)).startswith("inputs fit in L2")


def test_rooflines_from_phase_times():
    """Per-phase roofline entries: algorithmic work / time per launch, the
    dominant phase first, and a traffic figure only while its source matches."""
    import bench
    import workloads

    w = workloads.config("c2")
    K = 10
    ph = {name: {"ms": 0.0, "count": 0, "kernels": 0} for name in bench.PHASES}
    ph["overlap"] = {"ms": 13.0, "count": 10, "kernels": 10}   # 1.3 ms per launch
    ph["taylor"] = {"ms": 4.0, "count": 10, "kernels": 10}
    ph["qr"] = {"ms": 2.6, "count": 2, "kernels": 2}
    roofs = bench.rooflines(w, ph, "bf16", K)
    assert [r["phase"] for r in roofs] == ["overlap", "taylor", "qr"]
    ov = roofs[0]
    per = bench.algorithmic_per_walker(w)["overlap"]
    assert per == 8 * 25 ** 3
    assert bench.algorithmic_per_walker(w)["theta"] == 8 * (300 - 25) * 25 * 25
    assert abs(ov["achieved"] - per * 512 / 1.3e-3 / 1e12) < 1e-12
    # the bf16 mixed path keeps the elimination and Gram-Schmidt on the FP64 pipe
    assert ov["bound"] == "alu" and abs(ov["frac"] - ov["achieved"] / bench.FP64_PEAK_TFLOPS) < 1e-12
    assert roofs[1]["bound"] == "tensor"
    assert roofs[2]["bound"] == "alu" and roofs[2]["kernel"] == "k_mgs"
    # the opt-in -f32lu path: the elimination against the FP32 pipe, the
    # Gram-Schmidt sweep against HBM bandwidth
    r32 = bench.rooflines(w, ph, "bf16-f32lu", K)
    assert abs(r32[0]["frac"] - r32[0]["achieved"] / bench.FP32_PEAK_TFLOPS) < 1e-12
    qr = r32[2]
    pk, _ = bench.peaks()
    assert qr["bound"] == "hbm" and qr["unit"] == "GB/s" and qr["kernel"] == "k_mgs_f32"
    assert abs(qr["achieved"] - bench.bytes_per_walker(w, "bf16-f32lu")["qr"] * 512 / 1.3e-3 / 1e9) < 1e-9
    assert abs(qr["frac"] - qr["achieved"] / pk["hbm_gbs"]) < 1e-12
    assert set(bench.PRECISIONS) == {"fp64", "tf32", "bf16", "tf32-f32lu", "bf16-f32lu",
                                     "tf32-f64theta", "bf16-f64theta"}
    # Theta = Phi S^-1: FP32 from the float64 S^-1 on the default mixed path
    # (against HBM: it reads the float64 S^-1), float64 on -f64theta
    ph_t = dict(ph, theta={"ms": 0.5, "count": 10, "kernels": 10})
    th = [r for r in bench.rooflines(w, ph_t, "bf16", K) if r["phase"] == "theta"][0]
    assert th["bound"] == "hbm" and th["kernel"] == "k_theta_rows_f32"
    b = bench.bytes_per_walker(w, "bf16")["theta"]
    assert b == 2 * 25 * 300 * 8 * 2 + 25 * 25 * 16 + 2 * 25 * 304 * 2
    th64 = [r for r in bench.rooflines(w, ph_t, "bf16-f64theta", K) if r["phase"] == "theta"][0]
    assert th64["bound"] == "alu" and th64["kernel"] == "k_theta_rows"
    assert abs(sum(r["share_of_step"] for r in roofs) - 1.0) < 1e-12
    # a recorded traffic figure counts only for the source it was taken from
    saved = dict(bench.TRAFFIC)
    try:
        bench.TRAFFIC["overlap"] = {"bytes": 1.0e8, "sha": bench.source_sha("walker_f64.cu")}
        assert bench.rooflines(w, ph, "bf16", K)[0]["traffic"] == 1.0e8
        # the captures are of the BF16 step: another precision runs other kernels
        assert bench.rooflines(w, ph, "tf32", K)[0]["traffic"] is None
        bench.TRAFFIC["overlap"] = {"bytes": 1.0e8, "sha": "0" * 64}
        assert bench.rooflines(w, ph, "bf16", K)[0]["traffic"] is None
        # an entry may pin one kernel's own text instead of the whole file
        sig = "__global__ void __launch_bounds__(OV_T) k_overlap(OverlapArgs a)"
        fsha = bench.function_sha("walker_f64.cu", sig)
        assert fsha is not None and fsha != bench.source_sha("walker_f64.cu")
        bench.TRAFFIC["overlap"] = [{"bytes": 2.0e8, "function": sig, "sha": "1" * 64},
                                    {"bytes": 3.0e8, "function": sig, "sha": fsha}]
        assert bench.rooflines(w, ph, "bf16", K)[0]["traffic"] == 3.0e8
        assert bench.function_sha("walker_f64.cu", "no such kernel") is None
    finally:
        bench.TRAFFIC.clear()
        bench.TRAFFIC.update(saved)
