"""Host-side planning (no GPU): the cost model's per-segment strategy choice.

The planner estimates each pass's device time on GB300 from measured rates
(streaming tile / sweep / coset passes near the copy bandwidth, scattered
single-amplitude reads at a 64-byte DRAM access each, integer work per step
for non-affine gathers) and picks, per circuit segment, tile passes in place,
one gather pass, or a mix (Sec. 2i: sequential steps processed together).
These tests pin where the choice lands and where it flips.
"""
from collections import Counter

import numpy as np
import pytest

from paper_quant_ph_0308158_gb300 import plan_circuit_ex, workloads as W


def _plan(cfg_or_M, dtype=None, steps=None, **kw):
    if isinstance(cfg_or_M, dict):
        M, dtype, steps = cfg_or_M["M"], cfg_or_M["dtype"], cfg_or_M["steps"]
    else:
        M = cfg_or_M
    kw.setdefault("canonicalize", False)
    return plan_circuit_ex(M, dtype, steps, **kw)


def test_cnot_circuit_is_one_coset_gather():
    r = _plan(W.config_cnot(28))
    assert r["variants"] == ["coset"]
    # without a second buffer it stays in place
    r = _plan(W.config_cnot(28), scratch=False)
    assert set(r["variants"]) == {"tile"} and len(r["variants"]) > 10
    # with coset tiles off the affine gather reads scattered rows and is
    # charged accordingly (still one pass, still cheaper than ~48 tile passes)
    r2 = _plan(W.config_cnot(28), coset=False)
    assert r2["variants"] == ["affine"]
    assert r2["stats"]["est_ms"] > 3 * _plan(W.config_cnot(28))["stats"]["est_ms"]


@pytest.mark.parametrize("jit,variant", [(True, "compiled"), (False, "sliced")])
def test_mixed_circuit_is_one_gather(jit, variant):
    r = _plan(W.config_mixed_m28(), jit=jit)
    assert r["variants"] == [variant]


def test_hybrid_circuit_mixes_strategies_and_beats_both_pure_plans():
    cfg = W.config_hybrid()
    # without compiled kernels the register part becomes a short interpreted
    # gather; with them, passes over the register's tile that evaluate the
    # compiled steps (closed passes: the register steps change only tile bits)
    for jit, first in ((False, {"sliced"}), (True, {"closed"})):
        auto = _plan(cfg, jit=jit)
        gather = _plan(cfg, jit=jit, strategy="gather")
        tile = _plan(cfg, jit=jit, strategy="inplace")
        c = Counter(auto["variants"])
        assert c["coset"] == 1 and set(c) - {"coset"} == first
        assert auto["variants"][-1] == "coset"
        est = auto["stats"]["est_ms"]
        assert est < gather["stats"]["est_ms"] and est < tile["stats"]["est_ms"]
        # the tile passes cover register steps only, the coset gather the
        # CNOT layer (plus any NOT/CNOT steps that end the register part)
        ends = auto["pass_ends"]
        cut = int(ends[-2])
        assert 250 <= cut <= 300 and int(ends[-1]) == 1300
        assert sorted(auto["order"][:cut].tolist()) == list(range(cut))
        assert auto["order"][cut:].tolist() == list(range(cut, 1300))


def _chain_circuit(M, groups, seed):
    """groups of 9 Toffolis whose targets are 9 distinct high bits (cycling
    over three disjoint sets) and whose controls include the previous group's
    targets, so no step of a group commutes into another group's tile."""
    rng = np.random.default_rng(seed)
    sets = [list(range(4 + 9 * g, 13 + 9 * g)) for g in range(3)]
    rows = []
    prev = [0, 1, 2]
    for g in range(groups):
        tg = sets[g % 3]
        for t in tg:
            c = [int(x) for x in rng.choice([b for b in prev if b != t], size=2, replace=False)]
            m = (1 << c[0]) | (1 << c[1])
            rows.append((t, m, m))
        prev = tg
    return W.make_steps(rows)


@pytest.mark.parametrize("dtype,jit", [(np.complex128, True), (np.complex128, False), (np.complex64, True)])
def test_choice_flips_where_the_estimates_cross(dtype, jit):
    """Circuits needing p tile passes for p = 1..12: AUTO keeps in-place
    passes (tile passes, or closed passes where those are estimated cheaper)
    while they are estimated cheaper than one gather and switches to the
    gather after that, once."""
    M = 31
    picks = []
    for p in range(1, 13):
        steps = _chain_circuit(M, p, p)
        tile = _plan(M, dtype, steps, strategy="inplace", jit=jit)
        assert tile["variants"].count("tile") + tile["variants"].count("closed") == p
        gather = _plan(M, dtype, steps, strategy="gather", jit=jit)
        auto = _plan(M, dtype, steps, jit=jit)
        want = "tile" if tile["stats"]["est_ms"] <= gather["stats"]["est_ms"] else "gather"
        got = "tile" if set(auto["variants"]) <= {"tile", "closed"} else "gather"
        assert got == want, (p, auto["variants"])
        assert auto["stats"]["est_ms"] <= min(tile["stats"]["est_ms"], gather["stats"]["est_ms"]) * (1 + 1e-12)
        picks.append(got)
    flip = picks.index("gather")
    assert 2 <= flip <= 11 and picks[flip:] == ["gather"] * (12 - flip), picks


def test_auto_is_never_estimated_slower_than_a_pure_plan():
    for seed in range(20):
        rng = np.random.default_rng(seed)
        M = int(rng.integers(12, 30))
        L = int(rng.integers(10, 600))
        parts = [W.cnot_circuit(M, L, seed), W.mixed_circuit(M, L // 3 + 1, seed),
                 W.local_mixed_circuit(M, L // 2 + 1, seed, min(12, M))]
        steps = np.concatenate([parts[i] for i in rng.permutation(3)])
        for dtype in (np.complex64, np.complex128):
            auto = _plan(M, dtype, steps, jit=bool(seed & 1))
            for s in ("inplace", "gather"):
                other = _plan(M, dtype, steps, strategy=s, jit=bool(seed & 1))
                assert auto["stats"]["est_ms"] <= other["stats"]["est_ms"] * (1 + 1e-12)


def _changed_bits(M, steps, rows=1 << 16, seed=5):
    """The bits a circuit's row map changes, from sampled rows of the oracle's
    single-row evaluation (enough rows to see every changed bit here)."""
    import oracle
    r = np.random.default_rng(seed).integers(0, 1 << M, size=rows, dtype=np.uint64)
    return int(np.bitwise_or.reduce(oracle.source_rows(M, steps, r).astype(np.uint64) ^ r))


def test_adder_m32_in_place_is_one_closed_pass():
    """With compiled kernels and the circuit's changed-bit set known, the
    M = 32 adder in place is one closed pass, estimated near its measured
    11.8 ms (without probabilities); without compiled kernels it needs
    dozens of tile passes."""
    cfg = W.config_adder_m32()
    delta = _changed_bits(32, cfg["steps"])
    assert bin(delta).count("1") == 12
    r = _plan(cfg, strategy="inplace", scratch=False, jit=True, closed_delta=delta)
    assert r["variants"] == ["closed"]
    assert 10.0 < r["stats"]["est_ms"] < 14.0
    t = _plan(cfg, strategy="inplace", scratch=False, jit=False)
    assert set(t["variants"]) <= {"tile", "sweep"} and len(t["variants"]) > 30


@pytest.mark.parametrize("dtype,kmax", [(np.complex64, 14), (np.complex128, 13)])
def test_closed_pass_needs_the_changed_bits_to_fit_a_tile(dtype, kmax):
    """One closed pass covers a whole circuit only while the bits it changes
    fit one tile (14 bits of complex64, 13 of complex128): a circuit whose
    targets fill the low kmax bits is one pass, one whose targets fill kmax + 1
    bits needs more."""
    M = 24
    for width, one_pass in ((kmax, True), (kmax + 1, False)):
        steps = W.local_mixed_circuit(M, 300, 3, width)
        delta = _changed_bits(M, steps)
        assert delta == (1 << width) - 1
        r = _plan(M, dtype, steps, strategy="inplace", scratch=False, jit=True, closed_delta=delta)
        if one_pass:
            assert r["variants"] == ["closed"]
        else:
            assert len(r["variants"]) >= 2
