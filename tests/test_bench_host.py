"""Host-side accounting of bench.py (CPU): the counts and byte figures its roofline lines are
built from, against brute force over the Fourier indices."""
import itertools
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def distinct_brute(dims):
    """Fourier slices of a real tensor up to conjugation, taking the first half (and the
    middle) of the last mode: the slices whose SVD the t-SVT computes."""
    modes = dims[2:]
    nh = modes[-1]
    seen, count = set(), 0
    for k in itertools.product(*[range(n) for n in modes]):
        if k[-1] > nh // 2:
            continue
        partner = tuple((-x) % n for x, n in zip(k, modes))
        if partner in seen:
            continue
        seen.add(k)
        count += 1
    return count


@pytest.mark.parametrize("dims", [(4, 4, 1), (4, 4, 7), (4, 4, 8), (2, 2, 100), (2, 2, 3, 60),
                                  (2, 2, 4, 6), (2, 2, 1, 5), (2, 2, 3, 2, 40), (2, 2, 2, 2, 2),
                                  (2, 2, 2, 4, 2, 6), (2, 2, 3, 3, 3, 3), (2, 2, 8, 8, 3)])
def test_distinct_slices_match_brute_force(dims):
    assert bench.half_slices(dims) == distinct_brute(dims)


def test_distinct_slices_cover_the_spectrum():
    """Every Fourier slice is a distinct slice or the conjugate of one: the distinct count is
    (P + s) / 2 where s counts the self-conjugate slices (indices with 2k = 0 mod n on every
    mode)."""
    for dims in [(2, 2, 6), (2, 2, 5, 4), (2, 2, 3, 2, 40), (2, 2, 2, 3, 4, 5)]:
        modes = dims[2:]
        P = int(np.prod(modes))
        s = int(np.prod([1 + (n % 2 == 0) for n in modes]))
        assert bench.half_slices(dims) == (P + s) // 2


@pytest.mark.parametrize("dims", [(144, 176, 100), (288, 352, 3, 60), (144, 176, 3, 2, 40)])
def test_tube_bytes_is_two_spectra_and_three_real_tensors(dims):
    n12 = dims[0] * dims[1]
    stored = int(np.prod(dims[2:-1])) * (dims[-1] // 2 + 1)
    N = int(np.prod(dims))
    assert bench.tube_bytes(dims) == 2 * 8 * n12 * stored + 3 * 4 * N
    if dims == (144, 176, 100):
        assert bench.tube_bytes(dims) == pytest.approx(51.1e6, rel=1e-3)


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` (the oracle on the host cores) runs without a GPU and
    prints the contract's line for the reference implementation."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "lowrank", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "iters/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1


def test_equal_error_verdict():
    """Per tensor: within 1% (+1e-5) of the plain form's recovery error, or both at or below
    the FP32 floor 1e-4 of an exact recovery; the worst tensor and the misses are reported."""
    v = bench.equal_error_verdict([0.101, 4.8e-5, 0.2, 2e-4], [0.1, 3.5e-5, 0.1, 1e-4])
    assert v["missing"] == [2, 3] and v["tensors_meeting"] == 2 and not v["equal_error"]
    assert v["worst_tensor"] == 2 and abs(v["worst_ratio"] - 2.0) < 1e-12
    assert bench.equal_error_verdict([0.0505], [0.05])["equal_error"]
    assert not bench.equal_error_verdict([0.0506], [0.05])["equal_error"]


def test_tube_traffic_matches_its_profile():
    """The captured tube-pass traffic bench.py reports comes from the committed colour-video
    profile: same kernel sources, and DRAM bytes equal to the profile's read + write."""
    import re
    with open(os.path.join(ROOT, "profiles", "tube_tile_kernel_color_288x352x3x60.md")) as f:
        text = f.read()
    for path, sha in bench.TUBE_TRAFFIC["sources"].items():
        assert f"`{os.path.basename(path)}` sha256 `{sha}`" in text
    mb = [float(x) for x in re.findall(r"`dram__bytes_(?:read|write)\.sum` \| ([0-9.]+) MB", text)]
    assert len(mb) == 2
    assert abs(sum(mb) * 1e6 - bench.TUBE_TRAFFIC["bytes_per_launch"]) < 0.1e6
    assert bench.tube_traffic("video") is None
