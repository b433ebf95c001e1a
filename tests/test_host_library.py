"""Host-side logic of the CUDA library, runnable without a GPU: the C ABI
loads and exports every declared symbol, the symbolic chain derivation
reproduces the paper's printed counts and listing, and argument validation
rejects bad input before any device work."""
import ctypes
import itertools
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def smg():
    from paper_2506_21932_gb300 import build, smg as S
    build.build()
    return S


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "smg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(smg_\w+)\s*\(", hdr, flags=re.M)
    assert len(names) >= 10
    return names


def test_library_exports_every_declared_symbol(smg):
    L = smg.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert b"sm_103a" in L.smg_version()


def test_strerror_covers_every_status(smg):
    for s in range(8):
        assert smg.strerror(s) and "unknown" not in smg.strerror(s)


# ----------------------------------------------------------------------------
# Symbolic chain derivation (Sec. 4.3, Eq. 5-10, Table 2, Listing 1)
# ----------------------------------------------------------------------------

def pattern(name):
    cube = list(itertools.product((-1, 0, 1), repeat=3))
    return {
        "3d8c": list(itertools.product((0, 1), repeat=3)),
        "3d64c": list(itertools.product((-1, 0, 1, 2), repeat=3)),
        "3d7v": [o for o in cube if sum(map(abs, o)) <= 1],
        "3d27v": cube,
        "3d7": [o for o in cube if sum(map(abs, o)) <= 1],
        "3d19": [o for o in cube if sum(map(abs, o)) <= 2],
        "3d27": cube,
    }[name]


def test_chain_counts_match_table3(smg):
    gold = json.load(open(os.path.join(GOLD, "table3_chains.json")))
    for case in gold["cases"]:
        ch = smg.derive_chains(pattern(case["R"]), pattern(case["A"]), pattern(case["P"]))
        assert len(ch) == case["chains"], case


def test_chain_counts_of_the_build_combinations(smg):
    """The combinations the hierarchy uses: 3d27v on a 7-point fine matrix and
    on its 27-point coarse matrices, 3d8c on 7 points (all 56 chains of Table 2)."""
    assert len(smg.derive_chains(pattern("3d27v"), pattern("3d7"), pattern("3d27v"))) == 725
    assert len(smg.derive_chains(pattern("3d8c"), pattern("3d27"), pattern("3d8c"))) == 216
    # 3d8c keeps 7 points: only the 7 face/centre coarse offsets are reached
    ch = smg.derive_chains(pattern("3d8c"), pattern("3d7"), pattern("3d8c"))
    reached = sorted({c[3] for c in ch})
    assert reached == [4, 10, 12, 13, 14, 16, 22]


def test_listing1_chains_2d(smg):
    """2-D example of Fig. 3 / Listing 1: R, P 2d9 (vertex), A 2d5; the coarse
    neighbour (-1,+1) (index 2) receives exactly the listed five chains."""
    gold = json.load(open(os.path.join(GOLD, "listing1_chains.json")))
    p2d9 = [(dx, dy) for dx in (-1, 0, 1) for dy in (-1, 0, 1)]
    p2d5 = [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    ch = smg.derive_chains(p2d9, p2d5, p2d9, dim=2)
    got = sorted((r, a, q) for r, a, q, dj in ch if dj == gold["coarse_index"])
    assert got == sorted(tuple(c) for c in gold["chains_R_A_P"])
    # Eq. 10: for F_u at the left-up corner of C_i (fine offset (-1,+1)), the
    # reachable F_v of C_j = C_i + (-1,+1) are C_i + {(-2,1), (-1,1), (-1,2)}
    ru = p2d9.index((-1, 1))
    vs = sorted(tuple(p2d9[ru][t] + p2d5[a][t] for t in range(2)) for r, a, q, dj in ch
                if dj == gold["coarse_index"] and r == ru)
    assert vs == sorted(tuple(v) for v in gold["intersection_u_left_up"]["offsets_from_Ci"])


def test_chain_derivation_rejects_far_coarse_offsets(smg):
    far = [(-3, 0, 0), (0, 0, 0)]
    with pytest.raises(ValueError):
        smg.derive_chains(far, pattern("3d7"), pattern("3d27v"))


# ----------------------------------------------------------------------------
# Argument validation (returns before any device call)
# ----------------------------------------------------------------------------

def _setup_status(smg, dims, offs, block=1, opt=None):
    L = smg.lib()
    h = ctypes.c_void_p()
    flat = [c for o in offs for c in o]
    arr = (ctypes.c_int * len(flat))(*flat)
    d = (ctypes.c_int * 3)(*dims)
    o = ctypes.byref(opt) if opt is not None else None
    # a non-null dummy pointer: validation fails before it could be used
    return L.smg_setup(ctypes.byref(h), d, len(offs), arr, ctypes.c_void_p(16), block, o, None), h.value


def test_setup_rejects_bad_arguments(smg):
    from paper_2506_21932_gb300 import inputs as I
    assert _setup_status(smg, (0, 4, 4), I.OFF7) == (smg.EINVAL, None)
    assert _setup_status(smg, (4, 1025, 4), I.OFF7) == (smg.EINVAL, None)
    assert _setup_status(smg, (4, 4, 4), I.OFF7, block=2) == (smg.EINVAL, None)
    assert _setup_status(smg, (4, 4, 4), [(0, 0, 0), (0, 0, 1)]) == (smg.EINVAL, None)  # not symmetric
    assert _setup_status(smg, (4, 4, 4), [(0, 0, 1), (0, 0, -1)]) == (smg.EINVAL, None)  # no centre
    assert _setup_status(smg, (4, 4, 4), [(0, 0, 0), (0, 0, 2), (0, 0, -2)]) == (smg.EINVAL, None)
    assert _setup_status(smg, (4, 4, 4), [(0, 0, 0), (0, 0, 0)]) == (smg.EINVAL, None)  # duplicate
    bad = smg.Options(0, 0, 2, 0, 0, 1.0, 0, 0, 0)  # BF16 with 3 unknowns per point
    assert _setup_status(smg, (4, 4, 4), I.OFF7, block=3, opt=bad) == (smg.EINVAL, None)
    bad = smg.Options(0, 0, 0, 0, 0, 2.5, 0, 0, 0)  # relaxation weight outside (0, 2)
    assert _setup_status(smg, (4, 4, 4), I.OFF7, opt=bad) == (smg.EINVAL, None)
    bad = smg.Options(0, 0, 0, 2, 99, 1.0, 0, 0, 0)  # restart > 64
    assert _setup_status(smg, (4, 4, 4), I.OFF7, opt=bad) == (smg.EINVAL, None)
    bad = smg.Options(0, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, 3)  # warps per sweep strip outside 0..2
    assert _setup_status(smg, (4, 4, 4), I.OFF7, opt=bad) == (smg.EINVAL, None)
    L = smg.lib()
    assert L.smg_setup(None, None, 0, None, None, 1, None, None) == smg.EINVAL
    assert L.smg_vcycle(None, None, None, None) == smg.EINVAL
    assert L.smg_solve(None, None, None, 1e-9, 10, None, None, None) == smg.EINVAL
    assert L.smg_level_count(None) == 0


def test_setup_chain_tables_of_every_transfer(smg):
    """The chain tables the hierarchy set-up builds (product host code):
    Table 2's 1216 and 1728 chains for 3d8c / 3d19 / 3d64c and 3d8c / 3d27 /
    3d64c, the vertex and piecewise-constant pairs, and the x-y
    semi-coarsening pair (per dimension 2 x 2 = 4 matching (r, q) pairs in x
    and y for every stencil entry, 1 in z: 16 chains per fine entry), each
    with a 27-point coarse mask (7 for 3d8c on 7 points)."""
    off7, off19, off27 = pattern("3d7"), pattern("3d19"), pattern("3d27")
    assert smg.rap_chain_count(smg.C64C, off19) == (1216, 27)
    assert smg.rap_chain_count(smg.C64C, off27) == (1728, 27)
    assert smg.rap_chain_count(smg.C64C, off7) == (8 * 7 * 8, 27)
    assert smg.rap_chain_count(smg.FW27V, off27) == (2197, 27)
    assert smg.rap_chain_count(smg.FW27V, off7)[0] == 725
    assert smg.rap_chain_count(smg.PC8C, off7) == (56, 7)
    assert smg.rap_chain_count(smg.C16XY, off7) == (16 * 7, 27)
    assert smg.rap_chain_count(smg.C16XY, off27) == (16 * 27, 27)
    with pytest.raises(ValueError):
        smg.rap_chain_count(4, off7)
