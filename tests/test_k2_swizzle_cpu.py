"""Exhaustive CPU check of the tiled kernel's shared-memory layout: the
swizzle `K2Shape<d>::phys` and the warp-to-element map `K2Shape<d>::elem` are
read from the kernel source itself (their bodies are integer expressions whose
operator precedence is the same in C++ and Python) and checked for every
tile shape:

- phys is a bijection of the tile onto its shared-memory slots, and keeps
  every 16-byte unit (the element pair c0 = 2k, 2k + 1) whole and aligned;
- elem is a bijection of the CTA's element indices onto the tile;
- every warp's permuted read (the element orbit members sit at w o tau for
  all d! permutations tau) takes the minimum number of shared-memory
  wavefronts, 2 for 32 doubles;
- every warp of the tile copy (consecutive 16-byte units along the rows,
  as the copy loop assigns them) takes the minimum, 4 for 32 units.

A double occupies two of the 32 four-byte banks, so the wavefronts a warp
needs are the largest number of its accesses that fall on one of the 16
eight-byte bank pairs (address mod 16, in doubles)."""
import itertools
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1705_06661_gb300", "csrc", "ss_k2.cuh")


def _body(text: str, head: str) -> list:
    i = text.index(head) + len(head)
    j = text.index("\n  }", i)
    stmts = []
    for st in text[i:j].split(";"):
        st = re.sub(r"//[^\n]*", "", st).strip()
        if not st:
            continue
        if st.startswith("const int "):
            stmts.extend(p.strip() for p in st[len("const int "):].split(","))
        elif st.startswith("return "):
            stmts.append("_r = " + st[len("return "):])
        else:
            stmts.append(st)
    return stmts


def _shape(d: int):
    text = open(SRC).read()
    i = text.index(f"struct K2Shape<{d}> {{")
    block = text[i:text.index("\n};", i)]
    bl, nt = map(int, re.search(r"static constexpr int BL = (\d+), NT = (\d+);", block).groups())
    phys_code = "\n".join(_body(block, "phys(const int (&c)[4]) {"))
    elem_code = "\n".join(_body(block, "elem(int e, int (&w)[4]) {"))

    def phys(c):
        env = {"c": list(c) + [0] * (4 - len(c))}
        exec(phys_code, {}, env)
        return env["_r"]

    def elem(e):
        env = {"e": e, "w": [0, 0, 0, 0]}
        exec(elem_code, {}, env)
        return env["w"][:d]

    return bl, nt, phys, elem


def _wavefronts(slots):
    count = {}
    for p in slots:
        count[p % 16] = count.get(p % 16, 0) + 1
    return max(count.values())


@pytest.mark.parametrize("d", [2, 3, 4])
def test_swizzle_is_a_bijection_keeping_pairs(d):
    bl, nt, phys, _ = _shape(d)
    assert bl ** d == nt
    offs = list(itertools.product(range(bl), repeat=d))
    slots = [phys(c) for c in offs]
    assert sorted(slots) == list(range(nt))
    for c in offs:
        if c[0] % 2 == 0:
            p = phys(c)
            assert p % 2 == 0 and phys((c[0] + 1,) + c[1:]) == p + 1


@pytest.mark.parametrize("d", [2, 3, 4])
def test_warp_map_covers_the_tile(d):
    bl, nt, _, elem = _shape(d)
    assert sorted(tuple(elem(e)) for e in range(nt)) == sorted(itertools.product(range(bl), repeat=d))


@pytest.mark.parametrize("d", [2, 3, 4])
def test_permuted_reads_take_two_wavefronts(d):
    _, nt, phys, elem = _shape(d)
    for tau in itertools.permutations(range(d)):
        for w0 in range(0, nt, 32):
            reads = [phys([elem(e)[tau[k]] for k in range(d)]) for e in range(w0, w0 + 32)]
            assert _wavefronts(reads) == 2, (d, tau, w0)


@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("unit", [2, 1])
def test_tile_copy_takes_minimum_wavefronts(d, unit):
    bl, nt, phys, _ = _shape(d)
    cpr, cpt = bl // unit, nt // unit
    for c0 in range(0, cpt, 32):
        slots = []
        for c in range(c0, min(c0 + 32, cpt)):
            w, r = [(c % cpr) * unit], c // cpr
            for _ in range(1, d):
                w.append(r % bl)
                r //= bl
            p = phys(w)
            slots.extend(p + i for i in range(unit))
        assert _wavefronts(slots) == len(slots) // 16, (d, unit, c0)
