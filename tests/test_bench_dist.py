"""bench.py's multi-rank plumbing on CPU: world size 2 over gloo, each rank
reports its own step time and every rank gets the maximum (the bench's
whole-job time); the reference arm only prints on rank 0."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    d = bench.dist_init("gloo")
    got = bench.reduce_max(10.0 + rank * 5.0, d, "cpu")
    bench.barrier(d)
    q.put((rank, got, bench.dist_env()))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert [o[2] for o in out] == [(2, 0, 0), (2, 1, 1)]


def test_roofline_bounds_and_traffic_come_from_the_right_summaries():
    # the apply graph is HBM-bound; the FP64 GEMM has no traffic summary of
    # its own and takes the DGEMM rate measured in the run when there is one
    import bench
    peaks = {"hbm_gbs": 6785.9, "bf16_tflops": 1911.6, "bf16_tflops_sustained": 1736.6}
    assert bench.kernel_bound("apply", "mixed", peaks)[0] == "hbm"
    assert bench.kernel_bound("k_gemm", "mixed", peaks)[0] == "tensor"
    assert bench.kernel_bound("k_gemm", "fp64", peaks)[:3] == ("alu", "TFLOP/s", 1.25)
    assert bench.kernel_bound("k_gemm", "fp64", dict(peaks, fp64_tflops=1.1))[:3] == ("alu", "TFLOP/s", 1.1)
    assert bench.traffic_from_profiles("k_gemm", "fp64") is None
    prof = {"apply": dict(launches=4, ms=2.0, flops=0.0, bytes=4 * 1.181e9),
            "k_gemm": dict(launches=10, ms=1.0, flops=1e10, bytes=0.0)}
    r = bench.roofline(prof, "mixed", peaks)
    assert r["kernel"] == "apply" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(4 * 1.181e9 / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6785.9, rel=1e-3)
