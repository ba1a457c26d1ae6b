"""Host-side basis plan of libkpm (CPU only), checked against plain combinatorics.

The S^z sectors of Sec. 2 (states with a fixed number of up spins) are ranked
in colex order, rank = sum_j C(p_j, j+1) over the set-bit positions p_j.  The
test checks the binomial table, each sector's hi-blocks with their first
ranks, each tile's first and last hi-block, and the list kernel's tile sizes."""
import math
import os
import shutil
import subprocess

import pytest

from paper_2104_13218_gb300 import _lib

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def colex_rank(s: int) -> int:
    r, j = 0, 0
    p = 0
    while s:
        if s & 1:
            j += 1
            r += math.comb(p, j)
        s >>= 1
        p += 1
    return r


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    _lib.lib()  # builds libkpm.so if needed
    libdir = os.path.join(ROOT, "paper_2104_13218_gb300", "_build")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_dump")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I" + os.path.join(ROOT, "include"),
                    "-I" + os.path.join(ROOT, "paper_2104_13218_gb300", "csrc"), "-I" + cuda_inc,
                    os.path.join(HERE, "host", "plan_dump.cpp"), "-o", exe, "-L" + libdir, "-lkpm",
                    "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return [line.split() for line in out.splitlines()]


def test_binomial_table(dump):
    rows = [r for r in dump if r[0] == "binom"]
    assert len(rows) == 65 * 66 // 2
    for _, n, k, v in rows:
        assert int(v) == math.comb(int(n), int(k))


def _plans(dump):
    plans, cur = [], None
    for r in dump:
        if r[0] == "plan":
            cur = {"N": int(r[1]), "ts": int(r[2]), "L": int(r[3]), "sectors": [], "blocks": [],
                   "tiles": []}
            plans.append(cur)
        elif r[0] == "sector":
            cur["sectors"].append([int(v) for v in r[1:]])
        elif r[0] == "block":
            cur["blocks"].append([int(v) for v in r[1:]])
        elif r[0] == "tile":
            cur["tiles"].append([int(v) for v in r[1:]])
    return plans


def test_hi_blocks_and_tiles(dump):
    plans = _plans(dump)
    assert len(plans) == 6 * 4
    for p in plans:
        N, L, ts = p["N"], p["L"], p["ts"]
        sectors = p["sectors"]
        n_blocks = len(p["blocks"])
        for i, (s, k, dim, row0, hb0, t0, t1) in enumerate(sectors):
            assert dim == (2 ** N if k < 0 else math.comb(N, k))
            tiles = p["tiles"][t0:t1]
            # tiles cover the sector's ranks in order, each at most ts states
            assert sum(t[3] for t in tiles) == dim
            assert all(t[2] == j * ts and t[1] == row0 + t[2] and t[6] == s for j, t in enumerate(tiles))
            if k < 0:
                continue
            hb1 = next((x[4] for x in sectors[i + 1:] if x[1] >= 0), n_blocks)
            blocks = p["blocks"][hb0:hb1]
            # hi-blocks: every high pattern that can hold k bits, in increasing order,
            # starting at the colex rank of its smallest state
            his = [h for h in range(2 ** (N - L)) if 0 <= k - bin(h).count("1") <= L]
            assert [b[1] for b in blocks] == his
            for _, hi, off in blocks:
                c = k - bin(hi).count("1")
                assert off == colex_rank((hi << L) | ((1 << c) - 1))
            offs = [b[2] for b in blocks]

            def block_of(rank):
                j = max(q for q in range(len(offs)) if offs[q] <= rank)
                return hb0 + j
            for t in tiles:
                assert t[4] == block_of(t[2])
                assert t[5] == block_of(t[2] + t[3] - 1)


def test_list_tile_states(dump):
    for _, gpw, rows, t in (r for r in dump if r[0] == "lts"):
        gpw, rows, t = int(gpw), int(rows), int(t)
        assert t % gpw == 0 and t >= max(16, gpw)
        assert -(-rows // t) <= (1 << 22)
