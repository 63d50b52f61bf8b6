"""Host logic of libsl1m that needs no GPU: the stream-K work split and the
k-d granule order (through the library's host-only entry points)."""
import numpy as np
import pytest

from paper_1310_2078_gb300 import synth

G = 64


@pytest.fixture(scope="module")
def sl1m():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_2078_gb300 import sl1m as s
    return s


CASES = [([1], [1], 608), ([5], [16], 608), ([79], [1024], 456), ([794], [16384], 456),
         ([3, 0, 7, 2], [10, 5, 0, 33], 17), ([1, 1, 1], [1, 1, 1], 1000), ([12], [7], 5)]


@pytest.mark.parametrize("nb,ns,cmax", CASES)
def test_stream_k_plan_covers_every_unit_once(sl1m, nb, ns, cmax):
    pv = sl1m.plan_preview(nb, ns, cmax)
    U = sum(a * b for a, b in zip(nb, ns))
    C = max(1, min(cmax, U))
    assert pv["n_units"] == U and pv["n_ctas"] == C
    # independent recomputation: CTA c takes [cU/C, (c+1)U/C)
    lo = [(U * c) // C for c in range(C)]
    hi = [(U * (c + 1)) // C for c in range(C)]
    gb, slot = 0, 0
    u0 = 0
    for a, b in zip(nb, ns):
        for blk in range(a):
            s, e = u0 + blk * b, u0 + (blk + 1) * b
            ctas = [c for c in range(C) if lo[c] < e and hi[c] > s] if b else []
            assert pv["first_slot"][gb] == slot
            if ctas:
                assert pv["first_cta"][gb] == ctas[0]
                assert pv["n_ctas_blk"][gb] == len(ctas) == ctas[-1] - ctas[0] + 1
            else:
                assert pv["n_ctas_blk"][gb] == 0
            slot += len(ctas)
            gb += 1
        u0 += a * b
    assert pv["n_slots"] == slot
    # every unit is in exactly one CTA range
    assert lo[0] == 0 and hi[-1] == U and all(hi[c] == lo[c + 1] for c in range(C - 1))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cost_weighted_plan_balances_cost(sl1m, seed):
    """Units of unequal cost (clustered 3x tiles): every CTA gets total/C of
    the cost up to one unit, blocks stay consistent with the CTA ranges."""
    rng = np.random.default_rng(seed)
    nb, ns, cmax = [7, 3], [200, 57], 40
    U = 7 * 200 + 3 * 57
    cost = np.ones(U, np.float32)
    start = rng.integers(0, U - 300)
    cost[start:start + 300] = 3.0                       # a clustered run of costly units
    cost[rng.choice(U, 50)] = 1.6
    pv = sl1m.plan_preview(nb, ns, cmax, cost)
    cu = pv["cta_first_unit"]
    C = pv["n_ctas"]
    assert cu[0] == 0 and cu[-1] == U and np.all(np.diff(cu) >= 0)
    per = np.array([cost[cu[c]:cu[c + 1]].sum() for c in range(C)])
    assert per.max() <= cost.sum() / C + cost.max() + 1e-3
    # a uniform split would be much worse on this input
    uni = np.array([cost[(U * c) // C:(U * (c + 1)) // C].sum() for c in range(C)])
    assert per.max() < uni.max()
    # block tables agree with the CTA ranges
    gb, u0 = 0, 0
    for a, b in zip(nb, ns):
        for blk in range(a):
            s_, e_ = u0 + blk * b, u0 + (blk + 1) * b
            ctas = [c for c in range(C) if cu[c] < e_ and cu[c + 1] > s_]
            assert pv["first_cta"][gb] == ctas[0] and pv["n_ctas_blk"][gb] == len(ctas)
            gb += 1
        u0 += a * b


def test_cost_weighted_plan_has_no_empty_cta(sl1m):
    """Few units of very unequal cost: every CTA still gets a unit (a block's
    partial slots are those of all CTAs between its first and its last)."""
    cost = np.array([1, 9, 1, 1, 9, 9, 1, 1, 1, 9, 1, 1], np.float32)
    pv = sl1m.plan_preview([3], [4], 12, cost)
    cu = pv["cta_first_unit"]
    assert pv["n_ctas"] == 12 and np.all(np.diff(cu) >= 1)
    pv = sl1m.plan_preview([2, 1], [3, 4], 7, np.array([5, 1, 1, 1, 1, 1, 9, 1, 1, 1], np.float32))
    assert np.all(np.diff(pv["cta_first_unit"]) >= 1)


def test_plan_rejects_bad_arguments(sl1m):
    with pytest.raises(sl1m.SL1MError):
        sl1m.plan_preview([1], [-1], 4)
    with pytest.raises(sl1m.SL1MError):
        sl1m.plan_preview([1], [1], 0)


@pytest.mark.parametrize("n", [1, 63, 64, 65, 1000, 4097])
def test_granule_order_is_a_padded_permutation(sl1m, n):
    xy = np.random.default_rng(n).uniform(-1, 1, (n, 2))
    order = sl1m.granule_order(xy)
    assert len(order) == -(-n // G) * G
    real = order[order >= 0]
    assert sorted(real.tolist()) == list(range(n))
    pad = np.flatnonzero(order < 0)
    assert pad.size == len(order) - n
    assert pad.size == 0 or pad[0] == n       # padding only in the last granule


def test_granules_of_a_regular_grid_are_8x8_blocks(sl1m):
    lm = synth.regular_grid(64, 0.5)
    order = sl1m.granule_order(lm)
    delta = 1.0 / 64
    for g in range(len(order) // G):
        pts = lm[order[g * G:(g + 1) * G]]
        ext = np.ptp(pts, axis=0)
        assert np.allclose(ext, 7 * delta)


def test_granules_are_compact_for_uv_tracks(sl1m):
    w = synth.config2(n_side=32)
    order = sl1m.granule_order(w.uvw[:, :2])
    ext = []
    for g in range(len(order) // G):
        idx = order[g * G:(g + 1) * G]
        idx = idx[idx >= 0]
        ext.append(np.ptp(w.uvw[idx, :2], axis=0).max())
    rnd = np.random.default_rng(0).permutation(w.n_vis)
    ext_rnd = [np.ptp(w.uvw[rnd[g * G:(g + 1) * G], :2], axis=0).max()
               for g in range(w.n_vis // G)]
    # k-d granules are more than an order of magnitude tighter than random ones
    assert np.median(ext) < 0.1 * np.median(ext_rnd)


def test_granule_order_of_a_large_input_is_deterministic_and_compact(sl1m):
    """Above 2^16 points the top levels of the k-d split run on threads: the
    order is still a padded permutation, the same on every call, and made of
    compact boxes (each granule's extent far below a random granule's)."""
    xy = np.random.default_rng(11).uniform(-1, 1, (300_001, 2))
    a = sl1m.granule_order(xy)
    b = sl1m.granule_order(xy)
    assert np.array_equal(a, b)
    real = a[a >= 0]
    assert real.size == 300_001 and np.array_equal(np.sort(real), np.arange(300_001))
    gr = a[: (len(a) // G - 1) * G].reshape(-1, G)
    ext = np.ptp(xy[gr], axis=1).max(axis=1)
    assert np.median(ext) < 0.05


# ---- the FP32 layout the mixed kernels read (exact phase split, Sect. 3.1)

def _layout_restated(xyzw, order):
    """The layout from its definition, in numpy: per granule the centre is the
    middle of its members' bounding box and the extent half the box (rounded
    up by a relative 1e-7); every stored FP32 value is one rounding of an FP64
    quantity (hi = fl32(x), lo = fl32(x - hi)); a padding slot copies the last
    member of its granule with auxiliary value 0."""
    f32 = np.float32
    npad = len(order)
    ng = npad // G
    hi = np.zeros((npad, 4), f32)
    lo = np.zeros((npad, 4), f32)
    off = np.zeros((npad, 4), f32)
    offlo = np.zeros((npad, 4), f32)
    cen_hi = np.zeros((ng, 4), f32)
    cen_lo = np.zeros((ng, 4), f32)
    ext = np.zeros((ng, 4), f32)
    for g in range(ng):
        idx = order[g * G:(g + 1) * G]
        real = idx[idx >= 0]
        if real.size:
            c = xyzw[real, :3]
            mn, mx = c.min(axis=0), c.max(axis=0)
            cen = 0.5 * (mn + mx)
            ext[g, :3] = ((mx - mn) * 0.5000001).astype(f32)
            ref = real[-1]
        else:
            cen = np.zeros(3)
        cen_hi[g, :3] = cen.astype(f32)
        cen_lo[g, :3] = (cen - cen.astype(f32).astype(np.float64)).astype(f32)
        for t, o in enumerate(idx):
            i = g * G + t
            if o >= 0:
                v, aux = xyzw[o, :3], xyzw[o, 3]
            elif real.size:
                v, aux = xyzw[ref, :3], 0.0
            else:
                v, aux = cen, 0.0
            hi[i, :3] = v.astype(f32)
            lo[i, :3] = (v - v.astype(f32).astype(np.float64)).astype(f32)
            d = v - cen
            off[i, :3] = d.astype(f32)
            off[i, 3] = f32(aux)
            offlo[i, :3] = (d - d.astype(f32).astype(np.float64)).astype(f32)
    return dict(hi=hi, lo=lo, off=off, offlo=offlo, cen_hi=cen_hi, cen_lo=cen_lo, ext=ext)


def _pixels_xyzw(lm):
    r2 = (lm ** 2).sum(axis=1)
    n = np.sqrt(1.0 - r2)
    return np.column_stack([lm[:, 0], lm[:, 1], -r2 / (1.0 + n), 1.0 / n])


@pytest.mark.parametrize("side", ["pixels", "visibilities"])
def test_granule_layout_is_its_definition(sl1m, side):
    """The library's FP32 layout of the wide-field geometry (l, m to +-0.5,
    w-term significant) equals the definition restated in numpy, bit for bit,
    and satisfies what the exact phase split needs: hi + lo and off + offlo
    give the FP64 coordinate and offset to 2^-47 relative, and the extent
    bounds every member's |offset| per axis."""
    w = synth.config2(n_side=47)                 # 2,209 pixels: a padded last granule
    if side == "pixels":
        xyzw = _pixels_xyzw(w.lm)
        order = sl1m.granule_order(w.lm)
    else:
        xyzw = np.column_stack([w.uvw, np.ones(w.n_vis)])
        order = sl1m.granule_order(w.uvw[:, :2])
    got = sl1m.granule_layout(xyzw, order)
    want = _layout_restated(xyzw, order)
    for k in want:
        assert np.array_equal(got[k].view(np.uint32), want[k].view(np.uint32)), k
    real = order >= 0
    c = xyzw[order[real], :3]
    assert np.all(np.abs(got["hi"][real, :3].astype(np.float64) + got["lo"][real, :3] - c)
                  <= 2.0 ** -47 * np.abs(c) + 1e-300)
    g = np.flatnonzero(real) // G
    cen = got["cen_hi"][g, :3].astype(np.float64) + got["cen_lo"][g, :3]
    d = c - cen
    assert np.all(np.abs(got["off"][real, :3].astype(np.float64) + got["offlo"][real, :3] - d)
                  <= 2.0 ** -46 * np.abs(c).max())
    assert np.all(np.abs(d) <= got["ext"][g, :3])
    assert np.array_equal(got["off"][real, 3], xyzw[order[real], 3].astype(np.float32))
    assert np.all(got["off"][~real, 3] == 0.0)


def test_granule_layout_of_a_large_input_on_threads(sl1m):
    """Above 1,024 granules the layout runs on host threads: still the
    definition, bit for bit (checked on a sample of granules), and the same on
    every call."""
    rng = np.random.default_rng(5)
    lm = rng.uniform(-0.4, 0.4, (200_003, 2))
    xyzw = _pixels_xyzw(lm)
    order = sl1m.granule_order(lm)
    a = sl1m.granule_layout(xyzw, order)
    b = sl1m.granule_layout(xyzw, order)
    for k in a:
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
    ng = len(order) // G
    for g in np.concatenate([rng.choice(ng - 1, 40, replace=False), [ng - 1]]):
        sub = order[g * G:(g + 1) * G]
        want = _layout_restated(xyzw, sub)
        sl = slice(g * G, (g + 1) * G)
        for k in ("hi", "lo", "off", "offlo"):
            assert np.array_equal(a[k][sl].view(np.uint32), want[k].view(np.uint32)), (g, k)
        for k in ("cen_hi", "cen_lo", "ext"):
            assert np.array_equal(a[k][g].view(np.uint32), want[k][0].view(np.uint32)), (g, k)


def test_granule_layout_rejects_a_bad_order(sl1m):
    xyzw = _pixels_xyzw(np.random.default_rng(0).uniform(-0.3, 0.3, (70, 2)))
    good = np.concatenate([np.arange(70), -np.ones(58, int)]).astype(np.int32)
    sl1m.granule_layout(xyzw, good)
    for bad in (np.concatenate([np.arange(69), [3], -np.ones(58, int)]),   # repeated index
                np.concatenate([np.arange(69), [70], -np.ones(58, int)]),  # out of range
                good[:100]):                                                 # not a multiple of 64
        with pytest.raises(sl1m.SL1MError):
            sl1m.granule_layout(xyzw, np.asarray(bad, np.int32))
