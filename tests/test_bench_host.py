"""CPU checks of bench.py's host-side helpers: the workload description at
the grid actually run, and the DRAM traffic record of the numeric kernel,
which the bench line reports only while the numeric kernels' sources have the
digest the record was taken on."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as w  # noqa: E402
from paper_1801_03065_gb300 import build as pkg_build  # noqa: E402


def test_workload_name_states_the_grid_run():
    A, P = w.stencil3d_27pt(100, seed=1), w.aggregation(100, 3)
    assert bench.workload_name(A, P, 100) == bench.WORKLOAD
    assert "26,463,592 nnz" in bench.WORKLOAD and "1,000,000 x 39,304" in bench.WORKLOAD
    A, P = w.stencil3d_27pt(20, seed=1), w.aggregation(20, 3)
    name = bench.workload_name(A, P, 20)
    assert name.startswith("stencil27_20:") and "20^3 grid" in name
    assert "%s rows" % format(A.nrows, ",") in name and "%s nnz" % format(A.nnz, ",") in name
    assert "(%s x %s)" % (format(P.nrows, ","), format(P.ncols, ",")) in name


def _record(tmp_path, digest, traffic=123456789):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / "rec.txt").write_text("# comment: ignored\nkernel: k\ntraffic_bytes_per_launch: %d\nbuild_digest: %s\n"
                               % (traffic, digest))


def test_traffic_record_only_at_its_digest(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic_record("rec.txt") is None   # no file
    _record(tmp_path, pkg_build._digest(pkg_build.NUMERIC_SOURCES))
    assert bench.load_traffic_record("rec.txt") == {"traffic_bytes_per_launch": 123456789}
    _record(tmp_path, "0" * 64)
    assert bench.load_traffic_record("rec.txt") is None
    # the whole-library digest is not the numeric kernels' digest
    _record(tmp_path, pkg_build._digest())
    assert bench.load_traffic_record("rec.txt") is None


def test_numeric_digest_covers_only_its_sources(tmp_path, monkeypatch):
    """Changing a file outside the numeric kernels' sources keeps their digest;
    changing one of them changes it."""
    src = tmp_path / "csrc"
    src.mkdir()
    for n in pkg_build.NUMERIC_SOURCES + ["kks_symbolic.cu"]:
        (src / n).write_text("// " + n + "\n")
    monkeypatch.setattr(pkg_build, "CSRC", str(src))
    d0 = pkg_build._digest(pkg_build.NUMERIC_SOURCES)
    (src / "kks_symbolic.cu").write_text("// changed\n")
    assert pkg_build._digest(pkg_build.NUMERIC_SOURCES) == d0
    (src / "kks_numeric.cu").write_text("// changed\n")
    assert pkg_build._digest(pkg_build.NUMERIC_SOURCES) != d0


@pytest.mark.parametrize("flag", ["--sym-merge", "--stage-b", "--dense"])
def test_option_flags_parse(flag):
    args = bench.parse_args([flag, "0"])
    assert args.gpus == 1 and args.steps >= 1 and args.warmup >= 3
