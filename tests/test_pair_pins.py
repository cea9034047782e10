"""Pins of the oracle's paired-texel decoder (no GPU): hand-derived pairs from
the paper's data section (tests/golden/pair_codec.json), the per-cell and the
whole-array decoders against each other, and round trips through the input
generator's encoder."""

import json
import os

import numpy as np
import pytest

import synth
from oracle import pairs
from synth.pairs import encode_pairs, pairify

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pair_codec.json")


def _golden():
    return json.load(open(GOLDEN))


def _cells(rows):
    return np.array([[h0 | (h1 << 8) | (h2 << 16) | (m << 24) for h0, h1, h2, m in r] for r in rows],
                    dtype=np.uint32)


@pytest.mark.parametrize("dec", [pairs.decode_loop, pairs.decode])
def test_hand_derived_pairs_decode(dec):
    for case in _golden()["valid"]:
        t = np.array(case["texels"], dtype=np.uint16)
        assert (dec(t) == _cells(case["cells"])).all(), case["name"]


@pytest.mark.parametrize("val", [pairs.validate_loop, pairs.validate])
def test_hand_derived_invalid_pairs(val):
    for case in _golden()["invalid"]:
        t = np.array(case["texels"], dtype=np.uint16)
        assert val(t) == (False, case["first_bad"]), case["name"]
        with pytest.raises(ValueError):
            pairs.decode(t)
    for case in _golden()["valid"]:
        assert val(np.array(case["texels"], dtype=np.uint16)) == (True, None)


def test_odd_width_is_rejected():
    with pytest.raises(ValueError):
        pairs.decode(np.zeros((2, 3), np.uint16))


def _valid_cell(c):
    h0, h1, h2 = c & 0xFF, (c >> 8) & 0xFF, (c >> 16) & 0xFF
    return (h2 >= h1) if h1 > h0 else (h1 == 0 and h2 == 0)


def test_round_trip_through_the_generator_encoder():
    rng = np.random.default_rng(5)
    for seed, (W, H, f) in enumerate([(64, 48, 0.3), (2, 5, 0.9), (130, 17, 0.0), (40, 40, 1.0)]):
        cells, _ = synth.make_grid(W, H, seed=seed + 10, slab_frac=f)
        p = pairify(cells)
        assert (pairify(p) == p).all()
        t = encode_pairs(p)
        assert t.dtype == np.uint16 and t.shape == p.shape
        d = pairs.decode(t)
        assert (d == p).all()
        if W * H <= 4096:
            assert (pairs.decode_loop(t) == d).all()
        assert all(_valid_cell(int(c)) for c in d.ravel()[:: max(1, d.size // 500)])
        # pairs without any slab are left alone
        h0, h1, _, _ = synth.unpack_cells(cells)
        slab = h1 > h0
        plain = ~(slab[:, 0::2] | slab[:, 1::2])
        assert (p[:, 0::2][plain] == cells[:, 0::2][plain]).all()
        assert (p[:, 1::2][plain] == cells[:, 1::2][plain]).all()
    with pytest.raises(ValueError):
        encode_pairs(np.array([[synth.pack_cells(1, 5, 9, 0), synth.pack_cells(2, 0, 0, 0)]],
                              dtype=np.uint32))


def test_whole_array_decoder_equals_the_per_cell_one_on_random_texels():
    rng = np.random.default_rng(11)
    n_valid = 0
    for it in range(40):
        H, W = int(rng.integers(1, 9)), 2 * int(rng.integers(1, 9))
        t = np.zeros((H, W), np.uint16)
        for y in range(H):
            for k in range(W // 2):
                if rng.random() < 0.5:
                    t[y, 2 * k] = int(rng.integers(0, 256)) | (int(rng.integers(0, 8)) << 8)
                    t[y, 2 * k + 1] = int(rng.integers(0, 256)) | (int(rng.integers(0, 8)) << 8)
                    continue
                lo = int(rng.integers(0, 255))
                hi = int(rng.integers(lo + 1, 256))
                delta = int(rng.integers(0, hi - lo))
                t[y, 2 * k] = lo | ((0x80 | ((delta >> 4) << 3) | int(rng.integers(0, 8))) << 8)
                t[y, 2 * k + 1] = hi | ((0x80 | ((delta & 15) << 3) | int(rng.integers(0, 8))) << 8)
        assert pairs.validate(t) == pairs.validate_loop(t) == (True, None)
        assert (pairs.decode(t) == pairs.decode_loop(t)).all()
        n_valid += 1
        # one random corruption: both validators find the same first bad pair
        bad = t.copy()
        y, x = int(rng.integers(0, H)), int(rng.integers(0, W))
        bad[y, x] = int(rng.integers(0, 1 << 16))
        assert pairs.validate(bad) == pairs.validate_loop(bad)
    assert n_valid == 40


MUTANTS = [
    ("mid measured up from the floor",
     "mid = high - (16 * ((int(m[y, e]) >> 3) & 15) + ((int(m[y, o]) >> 3) & 15))",
     "mid = low + (16 * ((int(m[y, e]) >> 3) & 15) + ((int(m[y, o]) >> 3) & 15))"),
    ("nibbles swapped",
     "mid = high - (16 * ((int(m[y, e]) >> 3) & 15) + ((int(m[y, o]) >> 3) & 15))",
     "mid = high - (16 * ((int(m[y, o]) >> 3) & 15) + ((int(m[y, e]) >> 3) & 15))"),
    ("one material for the pair", "mat = int(m[y, x]) & 7", "mat = int(m[y, x - (x % 2)]) & 7"),
    ("odd cell's floor from its own texel", "h0, h1, h2 = low, mid, high",
     "h0, h1, h2 = int(v[y, x]), mid, high"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS)
def test_golden_pairs_catch_planted_decoder_mistakes(name, old, new):
    src = open(pairs.__file__).read()
    assert src.count(old) == 1, name
    ns = {}
    exec(compile(src.replace(old, new), "mutant", "exec"), ns)
    caught = False
    for case in _golden()["valid"]:
        t = np.array(case["texels"], dtype=np.uint16)
        try:
            got = ns["decode_loop"](t)
        except ValueError:
            caught = True
            break
        if not (got == _cells(case["cells"])).all():
            caught = True
            break
    assert caught, name
