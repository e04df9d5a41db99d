"""The piece schedule of calls that run in pieces from page-locked host buffers
(paper_2205_15311_gb300/csrc/jatam_pipe.h, host code): compiled here with the
host compiler and checked over many call sizes.

Invariants: the pieces cover the call exactly, in order, none empty; every piece
fits the per-piece list buffer (`per`); at most 8 pieces; the staggered form
(calls without the window) has one piece per two piece units (at least two),
equal but for a last one of a quarter; the paired form (calls with the window) falls
geometrically from the first piece to the last, at most 4 pieces; staged record
inputs give two equal halves; the overrides are honoured."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_15311_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "jatam_pipe.h"
int main()
{
    unsigned long long n, unit;
    int windowed, staged, form, pieces;
    while (std::scanf("%llu %llu %d %d %d %d", &n, &unit, &windowed, &staged, &form, &pieces) == 6) {
        jatam::PipeSchedule ps;
        const bool ok = jatam::pipe_schedule(n, unit, windowed != 0, staged != 0, form, pieces, &ps);
        std::printf("%d %zu %zu %d", ok ? 1 : 0, ps.pieces, ps.per, ps.stagger ? 1 : 0);
        for (size_t i = 0; i < ps.pieces; ++i) std::printf(" %zu", ps.sizes[i]);
        std::printf("\n");
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def schedule(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("pipe")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(cases):
        text = "".join(f"{n} {u} {int(w)} {int(s)} {f} {p}\n" for n, u, w, s, f, p in cases)
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
        res = []
        for line in out[: len(cases)]:
            v = [int(x) for x in line.split()]
            res.append({"ok": v[0] == 1, "pieces": v[1], "per": v[2], "stagger": v[3] == 1, "sizes": v[4:]})
        return res

    return run


UNIT = 1 << 22
SIZES = sorted({2 * UNIT, 2 * UNIT + 1, 3 * UNIT - 7, 1 << 24, (1 << 24) + 4_000_001, 10 ** 7, 10 ** 8,
                (1 << 26) + 7, 1 << 28, (1 << 28) + 12_345, 1 << 30, 3 << 30})


def _common(r, n):
    assert r["ok"]
    sizes = r["sizes"]
    assert sum(sizes) == n and len(sizes) == r["pieces"] and 1 <= r["pieces"] <= 8
    assert all(s > 0 for s in sizes) and max(sizes) <= r["per"]


def test_staggered_without_window(schedule):
    cases = [(n, UNIT, False, False, -1, 0) for n in SIZES]
    for (n, *_), r in zip(cases, schedule(cases)):
        _common(r, n)
        assert r["stagger"]
        s = r["sizes"]
        assert len(s) == max(2, min(8, n // (2 * UNIT)))
        assert all(x == s[0] for x in s[:-1]) and s[-1] <= s[0]
        # the last piece is about a quarter of the others
        assert abs(s[-1] - s[0] / 4) <= 8
    # all of S_{2,8}: two pieces, 80 / 20
    assert schedule([(1 << 24, UNIT, False, False, -1, 0)])[0]["sizes"] == [13421773, 3355443]


def test_paired_geometric_with_window(schedule):
    cases = [(n, UNIT, True, False, -1, 0) for n in SIZES]
    for (n, *_), r in zip(cases, schedule(cases)):
        _common(r, n)
        assert not r["stagger"]
        s = r["sizes"]
        assert len(s) == min(4, n // UNIT)
        assert all(a > b for a, b in zip(s, s[1:]))  # falling
        assert abs(s[0] / s[-1] - 8) < 0.01  # to an eighth
    assert schedule([(1 << 28, UNIT, True, False, -1, 0)])[0]["sizes"] == [143165576, 71582788, 35791394, 17895698]


def test_staged_inputs_two_halves(schedule):
    cases = [(n, UNIT, w, True, -1, 0) for n in SIZES for w in (False, True)]
    for (n, _, w, *_), r in zip(cases, schedule(cases)):
        _common(r, n)
        assert r["pieces"] == 2 and r["sizes"][0] - r["sizes"][1] in (0, 1)
        assert r["stagger"] == (not w)


@pytest.mark.parametrize("form", [0, 1, 2, 3])
@pytest.mark.parametrize("pieces", [0, 2, 3, 5, 8])
def test_overrides(schedule, form, pieces):
    cases = [(n, UNIT, w, s, form, pieces) for n in SIZES for w in (False, True) for s in (False, True)]
    for (n, _, w, s, *_), r in zip(cases, schedule(cases)):
        _common(r, n)
        assert r["stagger"] == bool(form & 1)
        if pieces:
            assert r["pieces"] <= pieces
            if not s and form & 2:
                assert r["pieces"] == pieces  # geometric sizes use every piece
