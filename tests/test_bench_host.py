"""Host-side checks of bench.py's accounting (no GPU): the profiling
workload subsets, the algorithmic cell-update count of a step, and the use
of a committed ncu profile's DRAM figure only while its kernel source is
unchanged."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_profiling_subsets():
    c = bench.make_case("config2", shots=4, nt=40)
    g = c.geom
    assert g.n_shots == 4 and int(g.nt.max()) == 40 and len(g.wavelet) == 40
    full = bench.make_case("config2")
    assert full.geom.n_shots == 64 and 3000 <= int(full.geom.nt.min()) and int(full.geom.nt.max()) <= 4000
    m = bench.make_case("marmousi")
    assert (m.nz, m.nx, m.geom.n_shots) == (221, 601, 30)


def test_step_cell_updates():
    """6 U per step, U = sum over shots of nt_s x padded window cells."""
    c = bench.make_case("config2")
    g, nb = c.geom, c.nb
    NZ = c.nz + 2 * nb
    U = sum(int(g.nt[s]) * (int(g.win_x1[s] - g.win_x0[s]) + 2 * nb) * NZ for s in range(g.n_shots))
    assert bench.algorithmic_cells(c) == 6 * U


def test_profile_traffic_needs_the_profiled_source(tmp_path, monkeypatch):
    kernel = "fwd_pair_kernel"
    cells = 24253680
    t = bench.profiled_traffic(kernel, cells)
    txt = open(os.path.join(ROOT, "profiles", f"{kernel}_config2.md")).read()
    assert ("kernel source sha256[:16]: `%s`" % bench.kernel_source_hash(kernel)) in txt
    assert t is not None and 8 * cells <= t <= 16 * cells
    # The same profile under another source hash is not used.
    fake = tmp_path / "profiles"
    fake.mkdir()
    (fake / f"{kernel}_config2.md").write_text(txt.replace(bench.kernel_source_hash(kernel), "0" * 16))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: "f" * 16)
    assert bench.profiled_traffic(kernel, cells) is None
