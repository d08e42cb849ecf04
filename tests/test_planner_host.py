"""The planner on the host (adj_layout_preview, no GPU): tiles partition the blocks into
class-uniform groups within the tile capacity, each range is ordered most expensive tile
first, and the ranges are balanced on the estimated run time."""

import numpy as np
import pytest

import synth
import paper_2505_23618_gb300 as adj


def capacity(w, h):
    return min(4096 // (w * h), 256)


@pytest.fixture(scope="module")
def mixed():
    wl = synth.uhd_mixed(seed=3, frames=2)
    return wl, adj.layout_preview(wl.tfs, wl.blocks, wl.total, n_sm=152)


def test_tiles_partition_the_blocks(mixed):
    wl, r = mixed
    by_off = {int(b["offset"]) // 16: b for b in wl.blocks}
    seen = []
    for t in r["tiles"]:
        assert t["list_begin"] % 4 == 0, "a tile's offset list starts on a 16-byte boundary"
        assert 1 <= t["nblk"] <= capacity(t["w"], t["h"])
        offs = r["list"][t["list_begin"]:t["list_begin"] + t["nblk"]]
        for o in offs:
            b = by_off[int(o)]
            assert (b["w"], b["h"], b["tf_h"], b["tf_v"]) == (t["w"], t["h"], t["tf_h"], t["tf_v"])
        seen.extend(int(o) for o in offs)
    assert sorted(seen) == sorted(by_off), "every block in exactly one tile"
    assert len(r["list"]) >= max(t["list_begin"] + t["nblk"] for t in r["tiles"]) + 4


def test_ranges_heavy_first_and_balanced(mixed):
    wl, r = mixed
    rb, c = r["range_begin"].astype(int), r["costs"]
    assert rb[0] == 0 and rb[-1] == len(r["tiles"]) and len(rb) == 153
    assert np.all(np.diff(rb) >= 0)
    sums = []
    for a, b in zip(rb[:-1], rb[1:]):
        seg = c[a:b]
        assert np.all(np.diff(seg) <= 1e-12), "a range runs its most expensive tiles first"
        sums.append(seg.sum())
    sums = np.array(sums)
    # cut on the cumulative cost: ranges differ by at most about two tiles' cost
    assert sums.max() - sums.min() <= 2 * c.max() + 1e-9
    assert abs(sums.mean() - c.sum() / 152) < 1e-9


def test_cost_model_orders_the_classes():
    rng = np.random.default_rng(2)
    tfs = [synth.Tf(n=4, core=0), synth.Tf(n=64, core=0), synth.random_post(rng, 64, 0, 32),
           synth.random_band(rng, 64, 0, [0, 1] * 6)]

    def one(w, h, th, tv, n):
        blocks = np.zeros(n, dtype=synth.BLOCK_DTYPE)
        blocks["offset"] = np.arange(n) * w * h
        blocks["w"], blocks["h"], blocks["tf_h"], blocks["tf_v"] = w, h, th, tv
        r = adj.layout_preview(tfs, blocks, n * w * h, n_sm=1)
        return r["costs"]

    small = one(4, 4, 0, 0, 256)[0]
    plain = one(64, 64, 1, 1, 1)[0]
    post = one(64, 64, 2, 2, 1)[0]
    band = one(64, 64, 3, 3, 1)[0]
    assert post > band > plain and post > small
    part = one(4, 4, 0, 0, 100)
    assert part[0] < small, "a partial tile costs less than a full one"


def test_preview_errors():
    tfs = [synth.Tf(n=8, core=0)]
    blocks = np.zeros(2, dtype=synth.BLOCK_DTYPE)
    blocks["w"] = blocks["h"] = 8
    blocks["offset"] = (0, 32)                      # the second block overlaps the first
    with pytest.raises(adj.AdjError) as e:
        adj.layout_preview(tfs, blocks, 128)
    assert e.value.name == "ADJ_ERR_INVALID_ARG"
    blocks["offset"] = (0, 64)
    blocks["h"][1] = 4                              # an 8-point transform on 4-row columns
    with pytest.raises(adj.AdjError) as e:
        adj.layout_preview(tfs, blocks, 128)
    assert e.value.name == "ADJ_ERR_PARAM_MISMATCH"
    blocks["h"][1] = 8
    with pytest.raises(adj.AdjError) as e:
        adj.layout_preview(tfs, blocks, 128, n_sm=0)
    assert e.value.name == "ADJ_ERR_INVALID_ARG"
    r = adj.layout_preview(tfs, blocks, 128, n_sm=4)
    assert len(r["tiles"]) == 1 and r["tiles"][0]["nblk"] == 2


def test_preview_rejects_blocks_out_of_range():
    tfs = [synth.Tf(n=8, core=0)]
    one = np.zeros(1, dtype=synth.BLOCK_DTYPE)
    one["w"] = one["h"] = 8
    # an offset whose end would overflow a signed 64-bit sum is past the end, not wrapped around
    one["offset"] = np.iinfo(np.int64).max - 15
    with pytest.raises(adj.AdjError) as e:
        adj.layout_preview(tfs, one, 1 << 20)
    assert e.value.name == "ADJ_ERR_INVALID_ARG" and "extends past" in str(e.value)
    one["offset"] = (1 << 20) - 48                   # ends 16 samples past total_coefs
    with pytest.raises(adj.AdjError) as e:
        adj.layout_preview(tfs, one, 1 << 20)
    assert "extends past" in str(e.value)
    one["offset"] = (1 << 20) - 64                   # ends exactly at total_coefs
    assert len(adj.layout_preview(tfs, one, 1 << 20)["tiles"]) == 1
    # more blocks than disjoint 16-sample blocks can fit is rejected before anything is read
    many = np.zeros(5, dtype=synth.BLOCK_DTYPE)
    many["w"] = many["h"] = 8
    many["offset"] = np.arange(5) * 64
    with pytest.raises(adj.AdjError) as e:
        adj.layout_preview(tfs, many, 64)
    assert e.value.name == "ADJ_ERR_INVALID_ARG" and "cannot fit" in str(e.value)
    assert adj.layout_preview(tfs, many, 5 * 64)["tiles"]["nblk"].sum() == 5


@pytest.mark.parametrize("rows,name", [
    (((0, 12, 8, 0, 0),), "ADJ_ERR_UNSUPPORTED_SIZE"),            # 12 is not a block side
    (((0, 8, 8, 0, 5),), "ADJ_ERR_INVALID_ARG"),                  # transform index out of range
    (((0, 8, 16, 0, 0),), "ADJ_ERR_PARAM_MISMATCH"),              # 16 rows, 8-point transform
    (((8, 8, 8, 0, 0),), "ADJ_ERR_MISALIGNED"),                   # offset not a multiple of 16
    (((-16, 8, 8, 0, 0),), "ADJ_ERR_MISALIGNED"),                 # negative offset
    (((0, 8, 8, 0, 0), (48, 8, 8, 0, 0)), "ADJ_ERR_INVALID_ARG"), # overlap
    (((4064, 8, 8, 0, 0),), "ADJ_ERR_INVALID_ARG"),               # past total_coefs
])
def test_block_validation_codes(rows, name):
    """adj_layout_preview runs the same block validation as adj_plan_set_blocks."""
    tfs = [synth.Tf(n=8, core=0), synth.Tf(n=16, core=1)]
    with pytest.raises(adj.AdjError) as e:
        adj.layout_preview(tfs, np.array(list(rows), dtype=synth.BLOCK_DTYPE), 4096)
    assert e.value.name == name


def test_preview_of_an_empty_list():
    r = adj.layout_preview([synth.Tf(n=8, core=0)], np.zeros(0, dtype=synth.BLOCK_DTYPE), 0)
    assert r["tiles"].size == 0 and r["costs"].size == 0
    assert list(r["range_begin"]) == [0]
    assert not r["list"].any()             # only the spare entries the kernel may over-read
