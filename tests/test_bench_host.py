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
    """A profile's DRAM bytes per update scale to the launch size while its
    recorded source hash is the current one, and are ignored otherwise."""
    cells = 24253680
    src_root = tmp_path / "paper_2403_17518_gb300" / "csrc"
    src_root.mkdir(parents=True)
    for kernel in ("fwd_pair_kernel", "adj_pair_kernel", "born_tma_kernel"):
        for f in bench.KERNEL_SOURCES[kernel]:
            (src_root / f).write_text(open(os.path.join(ROOT, "paper_2403_17518_gb300", "csrc", f)).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    prof = tmp_path / "profiles"
    prof.mkdir()
    for kernel in ("fwd_pair_kernel", "adj_pair_kernel", "born_tma_kernel"):
        h = bench.kernel_source_hash(kernel)
        (prof / f"{kernel}_config2.md").write_text(
            f"kernel source sha256[:16]: `{h}`\n\nDRAM bytes per cell update: 12.5\n")
        assert bench.profiled_traffic(kernel, cells) == 12.5 * cells
        # The same profile under another source hash is not used.
        (prof / f"{kernel}_config2.md").write_text(
            f"kernel source sha256[:16]: `{'0' * 16}`\n\nDRAM bytes per cell update: 12.5\n")
        assert bench.profiled_traffic(kernel, cells) is None
    assert bench.profiled_traffic("no_such_kernel", cells) is None


def test_committed_profiles_state_their_source_hash():
    """Every committed step-kernel profile names the source hash it was taken on."""
    import re

    for kernel in bench.KERNEL_SOURCES:
        path = os.path.join(ROOT, "profiles", f"{kernel}_config2.md")
        if os.path.exists(path):
            assert re.search(r"kernel source sha256\[:16\]:\s*`?[0-9a-f]{16}", open(path).read()), path
