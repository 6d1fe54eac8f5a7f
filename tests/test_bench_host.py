"""Host arithmetic of bench.py's roofline on CPU: the algorithmic bytes per
site it divides by the kernel time (the table of spinor, link and W bytes),
and the rule that ncu traffic is reported only for the kernel source the
counters were taken on."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

WILSON, BRILLOUIN, STAGGERED, WLAP, BLAP, WSUV, BSUV = range(7)


def test_algorithmic_bytes_per_site():
    # FP32, N_c = 3, N_v = 12: spinor in + out once, links once (Brillouin: 80 W)
    assert bench.alg_bytes_per_site(WILSON, 3, 12) == 2 * 12 * 4 * 3 * 8 + 4 * 9 * 8 == 2592
    assert bench.alg_bytes_per_site(STAGGERED, 3, 12) == 2 * 12 * 3 * 8 + 4 * 9 * 8 == 864
    assert bench.alg_bytes_per_site(BRILLOUIN, 3, 12) == 2 * 12 * 4 * 3 * 8 + 80 * 9 * 8 == 8064
    assert bench.alg_bytes_per_site(WILSON, 3, 12, clover=True) == 2592 + 288
    assert bench.alg_bytes_per_site(WLAP, 3, 12) == 2592
    assert bench.alg_bytes_per_site(WSUV, 3, 12) == 864
    assert bench.alg_bytes_per_site(BLAP, 3, 12) == 8064
    assert bench.alg_bytes_per_site(BSUV, 3, 12) == 2 * 12 * 3 * 8 + 80 * 9 * 8 == 6336
    # FP64 doubles everything; N_v = 1 leaves the link bytes alone
    assert bench.alg_bytes_per_site(WILSON, 3, 12, eb=8) == 2 * 2592
    assert bench.alg_bytes_per_site(STAGGERED, 3, 1) == 2 * 3 * 8 + 288


def _source_hash(csrc, files):
    import hashlib
    h = hashlib.sha256()
    for f in files + ("common.cuh",):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def test_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    # a copy of the kernel sources and a summary written for them: traffic is
    # read while the hash matches and withheld once a kernel source changes
    root = tmp_path / "repo"
    csrc = root / "paper_2112_14640_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2112_14640_gb300", "csrc"), csrc)
    (root / "profiles").mkdir()
    files = {"staggered": ("staggered.cuh",), "wilson": ("wilson.cuh", "clover.cuh")}
    for op, t in (("staggered", 1234567), ("wilson", 7654321)):
        (root / "profiles" / ("%s_kernel_16x16x16x32_nv12.md" % op)).write_text(
            "# summary\n\nkernel_source_sha256_16: %s\ntraffic_bytes_per_launch: %d\n"
            % (_source_hash(str(csrc), files[op]), t))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.ncu_traffic("staggered") == 1234567
    assert bench.ncu_traffic("wilson") == 7654321
    assert bench.ncu_traffic("brillouin") is None          # no summary
    with open(csrc / "staggered.cuh", "a") as f:
        f.write("\n// changed\n")
    assert bench.ncu_traffic("staggered") is None
    assert bench.ncu_traffic("wilson") == 7654321
    with open(csrc / "common.cuh", "a") as f:
        f.write("\n// changed\n")
    assert bench.ncu_traffic("wilson") is None
