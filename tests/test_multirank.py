"""World-size-2 runs of the bench's process-group code on the CPU (gloo,
rendezvous on 127.0.0.1): the barrier and the max-over-ranks timing helper,
and the reference arm launched as two ranks (rank 0 alone measures and
prints one line; rank 1 exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    e = dict(os.environ)
    e.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
             MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    return e


def _run_ranks(argv, world, timeout):
    port = _free_port()
    procs = [subprocess.Popen(argv, env=_env(r, world, port), stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, cwd=ROOT) for r in range(world)]
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=timeout)
            outs.append((p.returncode, out, err))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    return outs


_DIST = """
import sys
sys.path.insert(0, {root!r})
import bench
d = bench.Dist()
d.barrier()
m = d.max(10.0 * (d.rank + 1))
print("RESULT", d.rank, d.world, m, flush=True)
d.close()
"""


def test_dist_max_over_two_gloo_ranks():
    outs = _run_ranks([sys.executable, "-c", _DIST.format(root=ROOT)], 2, 180)
    for r, (rc, out, err) in enumerate(outs):
        assert rc == 0, err[-2000:]
        res = [l.split() for l in out.splitlines() if l.startswith("RESULT")]
        assert res and res[0][1:] == [str(r), "2", "20.0"], out


def test_reference_arm_two_ranks():
    argv = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
            "--warmup", "0"]
    outs = _run_ranks(argv, 2, 600)
    for rc, _, err in outs:
        assert rc == 0, err[-2000:]
    lines0 = [l for l in outs[0][1].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1][1].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    d = json.loads(lines0[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
