"""The multi-GPU bench path without GPUs: two gloo ranks on the CPU run the
same whole-job reduction bench.py uses (slowest rank's time, summed
cell-updates) and get independent replica seeds; the reference arm of a
non-zero rank exits without work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = bench.reduce_over_ranks(10.0 + rank, 100 * (rank + 1), 1.0 + 0.5 * rank, 7 * (rank + 1), world)
        q.put((rank, out, bench.replica_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    mp = pytest.importorskip("torch.multiprocessing")
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, out, seed in res:
        assert out == (11.0, 300.0, 1.5, 21.0)         # max time, summed cells over both ranks
    assert res[0][2] != res[1][2]                        # independent replicas


def test_reference_arm_of_a_nonzero_rank_does_nothing(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 3, 2
    assert bench.reference_arm(A()) == 0
    assert capsys.readouterr().out == ""


def test_step_roofline_arithmetic():
    """The whole-step roofline: the method's minimum bytes (8 B per box cell +
    44 B per domain cell in FP32; BF16 halves the state's bytes; physics adds
    the ID-field's read and write) and the five-pass design's (the pass bytes
    summed: 8 + 8 + 8 + 8 + 8 = 40 B per box cell, + 16 B per domain cell
    when the top-two field is stored), over the step time, against the peak."""
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
    import bench
    r = bench.step_roofline(1.0e8, 1.0e7, 2.0, 5000.0, True)
    assert r["minimum_bytes_per_step"] == 8.0e8 + 4.4e8
    assert abs(r["achieved_minimum_gbs"] - 1.24e9 / 2e-3 / 1e9) < 1e-9
    assert abs(r["frac_minimum"] - r["achieved_minimum_gbs"] / 5000.0) < 1e-15
    assert abs(r["minimum_bound_ms"] - 1.24e9 / 5e12 * 1e3) < 1e-12
    assert r["design_bytes_per_box_cell"] == 40.0
    assert r["design_bytes_per_step"] == 4.0e9
    assert bench.step_roofline(1.0e8, 1.0e7, 2.0, 5000.0, True, keep_field=True)["design_bytes_per_step"] == 4.0e9 + 1.6e8
    assert "design_bytes_per_step" not in bench.step_roofline(1.0e8, 1.0e7, 2.0, 5000.0, False)
    assert bench.step_roofline(1.0e8, 0.0, 2.0, 5000.0, False, state_bytes=2)["minimum_bytes_per_step"] == 4.0e8
    assert bench.step_roofline(1.0e8, 0.0, 2.0, 5000.0, False, physics=True)["minimum_bytes_per_step"] == 1.6e9


def test_kernel_roofline_takes_the_longest_launch():
    """The dominant pass is the one with the longest time per launch; the
    field pass counts one read of phi_p and one write of phi_c per box cell
    (plus 16 B per domain cell when it stores the top-two field), a tier pass
    8 B per box cell of its tier."""
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
    import bench
    tiers = [4.0e7, 6.0e7, 0, 0, 0]
    r = bench.kernel_roofline({"p_field": 0.5, "p_redist_xy[tier1]": 0.4, "k_bin": 0.01}, tiers, 1.0e8, 1.6e7,
                              5000, 6800.0)
    assert r["kernel"] == "p_field"
    assert r["algorithmic_bytes_per_launch"] == 8.0 * 1.0e8
    rk = bench.kernel_roofline({"p_field": 0.5}, tiers, 1.0e8, 1.6e7, 5000, 6800.0, keep_field=True)
    assert rk["algorithmic_bytes_per_launch"] == 8.0 * 1.0e8 + 16.0 * 1.6e7
    assert abs(r["frac"] - r["algorithmic_bytes_per_launch"] / 0.5e-3 / 1e9 / 6800.0) < 1e-12
    r = bench.kernel_roofline({"p_field": 0.3, "p_redist_xy[tier1]": 0.4}, tiers, 1.0e8, 1.6e7, 5000, 6800.0)
    assert r["kernel"] == "p_redist_xy[tier1]" and r["units_per_launch"] == 6.0e7
    assert r["algorithmic_bytes_per_launch"] == 8.0 * 6.0e7
    r = bench.kernel_roofline({"p_conv_xy[tier0]": 0.4}, tiers, 1.0e8, 1.6e7, 5000, 6800.0, state_bytes=2)
    assert r["algorithmic_bytes_per_launch"] == 6.0 * 4.0e7


def test_traffic_hash_ignores_comments_not_code():
    """The traffic figures are keyed to the pass kernels' code: a comment or
    layout change keeps the key, a code change does not."""
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
    import bench
    a = "int f(int x) { // doubles\n  return 2 * x; /* the\n result */ }\n"
    b = "int f(int x) {\n    return 2 * x;   // twice x\n}\n"
    c = "int f(int x) { return 3 * x; }"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
