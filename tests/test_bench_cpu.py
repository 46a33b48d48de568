"""The measurement harness on the CPU: the reference arm's JSON line (one
process and under torchrun with two ranks), the max-over-ranks timing of
the multi-GPU path on two gloo ranks, and the algorithmic-byte and launch
counts the bench reports."""
import json
import os
import socket
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _json_lines(out: str):
    return [json.loads(x) for x in out.splitlines() if x.startswith("{")]


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "0.3"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["unit"] == "TFLOP/s" and d["higher_is_better"] is True
    b, tau, bits = bench.SETTLED["water7500"]
    assert d["config"]["leaf"] == b and d["config"]["tau"] == tau and d["config"]["n"] == 7500
    assert d["config"]["tier_bits"] == bits
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_torchrun_prints_once():
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference"


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(1.5 + rank, dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got == {0: 2.5, 1: 2.5}
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25


def test_leaf_alg_bytes_and_launch_count():
    st = {"packed_leaves_a": 10, "packed_leaves_b": 6}
    # C written once plus the packed leaves read once (4 B per element)
    assert bench.leaf_alg_bytes(st, 1000.0 ** 2, 16, "f16x3") == 4e6 + 4 * 256 * 16
    # the FP32 SIMT kernel reads A itself
    assert bench.leaf_alg_bytes(st, 1000.0 ** 2, 16, "fp32") == 8e6
    # the launch list of one step at n = 7500, b = 64 (depth 7): k_leaf_norms,
    # k_pyramid_up x2, k_cull_root, k_cull_tier x6, k_cull_finish, four
    # grouping kernels, k_tile_cull, k_leaf_max, k_leaf_pack, k_leaf_tc
    assert bench.kernels_per_step(7, 64, "f16x3") == 19
    assert bench.kernels_per_step(7, 64, "fp32") == 17


def test_cpu_baseline_reports_model_and_single_thread_rate():
    import spamm_inputs as gen
    from oracle import oracle as O
    assert bench.cpu_model().strip() and "logical CPUs" in bench.cpu_model()
    A = gen.exp_decay(512, 0.9, seed=0)
    threads = O.threads()
    v1, desc = bench.cpu_sample_single_thread(A, 16, 1e-6, 0.2)
    assert v1 > 0 and "kept leaf products" in desc
    assert O.threads() == threads          # restored


def test_clipped_flops_and_passes():
    """Kept flops over the leaves' extents inside the matrix (the ragged last
    leaf row and column clipped), and the tensor-core passes per product
    under precision chosen by norm."""
    import numpy as np
    import spamm_inputs as gen
    from oracle import oracle as O
    n, b, tau = 100, 16, 0.0
    A = gen.uniform_dense(n, seed=3)
    nl = -(-n // b)
    ij = [(0, 0), (nl - 1, nl - 1), (nl - 1, 0)]
    # tau = 0 on a dense matrix: every K is kept
    ext = [min(b, n - k * b) for k in range(nl)]
    want = sum(2.0 * ext[I] * ext[J] * sum(ext) for I, J in ij)
    assert bench.clipped_flops(A, b, tau, ij) == want
    assert bench.mma_passes("f16x3", {"leaf_triples": 10, "hi_products": 10}) == 3.0
    assert bench.mma_passes("f16x3", {"leaf_triples": 10, "hi_products": 0}) == 1.0
    assert bench.mma_passes("tf32", {"leaf_triples": 10, "hi_products": 10}) == 1.0
    del np, O
