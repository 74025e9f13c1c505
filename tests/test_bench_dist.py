"""The bench's multi-process plumbing on CPU (gloo, world size 2): max-over-ranks timing
and the reference arm under torchrun (rank 0 alone reports, the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    d = bench.init_dist(world, "gloo")
    bench.barrier(d)
    m = bench.max_over_ranks(10.0 * (rank + 1), d)
    out.put((rank, m))
    d.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 20.0, 1: 20.0}


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "c1_m24", "--steps", "1", "--warmup", "0",
           "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_compact_results_fit_the_tail():
    """bench.py prints one JSON line whose last key, `results`, is a flat rounded summary of
    the whole measurement; it must stay short enough (< 1400 characters) to be read whole in
    the last 1500 characters of the line."""
    import json
    import bench
    tta = lambda s: {"seconds": s, "max_rel_err_vs_reference": 4.6123456e-13, "max_rho": 1.41234e-13,
                     "n_found": 40, "n_in_disk_reference": 40}
    solves = {"alg1": tta(49.812345), "alg2": tta(15.312345)}
    mixed = {"value": 12.512345, "time_to_all_eigenpairs": {"alg1": tta(6.1), "alg2": tta(6.1)},
             "band_solve_c64": {"avg_launch_ms": 33.8123, "achieved_tflops": 6.0912,
                                "peak_tflops": bench.FP32_PEAK_TFLOPS}}
    c4 = {"create_s": 12.3456, "lu_ms": 11111.123, "tta_s": 70.123, "max_rel_err_vs_reference": 3.1e-11,
          "max_rho": 8.1e-13, "refine_solves": 123, "n_found": 60, "n_in_disk_reference": 60}
    batch = {"speedup": 1.33333, "mixed_precision": {"speedup": 1.4012}}
    simple = {"seconds": 14.0768}
    sens = {"band_solve_adj_c128": {"frac": 0.6012345}}
    roof = {"frac": 0.632145, "hbm_frac": 0.0046123}
    cpu = {"all_cores_value": 1.7232707}
    out = bench.compact_results(solves, mixed, c4, batch, simple, sens, roof, cpu)
    txt = json.dumps({"results": out})
    assert len(txt) < 1400, len(txt)
    assert all(not isinstance(v, (dict, list)) for v in out.values())
    assert out["tta_alg1_c128_s"] == 49.8 and out["nf_alg2_mixed"] == "40/40"
    assert out["c4_nf"] == "60/60"
    assert out["mixed_solve_frac_fp32"] == bench.r3(6.0912 / bench.FP32_PEAK_TFLOPS)
