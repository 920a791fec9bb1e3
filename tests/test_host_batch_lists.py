"""The batch's work lists on the host: `host/batch_lists_host.cc` builds each list kind
with `batch_layout` (what hweno_batch_init uploads) for every block shape the batch
launches it with (the autotuner's four shapes, kb_dr's block, the ghost and split
lines, the flux tiles and the TMA-staged gradient tiles), decodes every (item, thread)
with the kernels' own `find_case` and `tile_pos`, and counts how often each position of
each case's launch region is reached: exactly once everywhere, on ragged grids, a single
4 x 4 case and 64 cases of mixed sizes (the ensemble's largest count of cases with
tensor maps), under AddressSanitizer and UBSan where g++ has them."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from test_host_residual2d import CSRC, HERE, ROOT, SANITIZE

KINDS_AND_SHAPES = 4 * 6 + 1 + 2 + 2 + 1  # tuned kinds x 4 shapes, kb_dr, ghost/split, flux tiles, TMA tiles


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is needed to compile the device code for the host")
    out = str(tmp_path_factory.mktemp("batch_lists") / "batch_lists_host")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-strict-aliasing", "-I" + os.path.join(HERE, "host"),
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", out,
           os.path.join(HERE, "host", "batch_lists_host.cc")]
    if subprocess.run(cmd + SANITIZE, capture_output=True).returncode != 0:
        subprocess.check_call(cmd)
    return out


def _sizes(name):
    if name == "single_4x4":
        return [(4, 4)]
    if name == "ragged_five":
        return [(37, 21), (16, 16), (64, 32), (5, 70), (33, 7)]
    rng = np.random.default_rng(91)
    return [(int(a), int(b)) for a, b in rng.integers(4, 97, size=(64, 2))]


@pytest.mark.parametrize("name", ["single_4x4", "ragged_five", "mixed_64"])
def test_every_position_once(exe, name):
    sizes = _sizes(name)
    args = [str(v) for s in sizes for v in s]
    out = subprocess.check_output([exe] + args, timeout=600).decode().split("\n")
    rows = [list(map(int, line.split())) for line in out if line.strip()]
    assert len(rows) == KINDS_AND_SHAPES
    for kind, bx, by, total, bad in rows:
        assert total >= len(sizes), (kind, bx, by)
        assert bad == 0, (kind, bx, by, bad)
