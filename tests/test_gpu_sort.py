"""Binning and sort: the GPU's tile lists and order are bit-exact against a
CPU replay of the integer key derivation from the GPU's own pixel boxes, and
the records and boxes match the oracle's FP64 decisions."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_05643_gb300 import binding as B
from paper_2505_05643_gb300 import render as R
from paper_2505_05643_gb300 import synth

from gpu_helpers import gpu_render, oracle_config

pytestmark = pytest.mark.gpu


def _tile_offsets(planes, tile):
    W = planes["size"][:, 0]
    H = planes["size"][:, 1]
    tx = (W + tile - 1) // tile
    ty = (H + tile - 1) // tile
    off = np.concatenate([[0], np.cumsum(tx * ty)])
    return off, tx


def _expected_records(geo, chunks_n, P):
    """(plane, gaussian) of each record in the order (chunk of 32, plane, gaussian)."""
    vis = geo["visible"] & (geo["box"][..., 0] <= geo["box"][..., 1]) & \
        (geo["box"][..., 2] <= geo["box"][..., 3])
    out = []
    n = vis.shape[1]
    for c in range((n + 31) // 32):
        for p in range(P):
            for g in range(c * 32, min(n, c * 32 + 32)):
                if vis[p, g]:
                    out.append((p, g))
    return out


def _edge_ambiguous(geo, planes, p, g, amb=1e-5):
    m = geo["m"][p, g]
    h = geo["h"][p, g]
    W, Hh = planes["size"][p]
    pu, pv = planes["pitch"][p].astype(np.float64)
    for c, hh, size, pitch in ((m[0], h[0], W, pu), (m[1], h[1], Hh, pv)):
        for edge in (c - hh, c + hh):
            k = edge / pitch + size / 2 - 0.5  # pixel-unit position of the edge
            if abs(k - np.rint(k)) * pitch <= amb * pitch * 2:
                return True
    return bool(geo["amb_plane"][p, g])


def _max_exponent(a, b, c, box, j0, j1, i0, i1):
    """FP64 max over the pixel centres of [j0, j1] x [i0, i1] of the weight
    exponent lw2 - t1^2 - t2^2 of a record (a = X, Y, r11, kappa; c = their
    low parts; b = r22, lw2, ...; X, Y relative to the box's first column and
    row): t1 = r11 (dx + kappa dy), t2 = r22 dy."""
    a, b, c = a.astype(np.float64), b.astype(np.float64), c.astype(np.float64)
    X, Y, kap = a[0] + c[0], a[1] + c[1], a[3] + c[2]
    bj0, bi0 = int(box[0] & 0xFFFF), int(box[1] & 0xFFFF)
    jj, ii = np.meshgrid(np.arange(j0, j1 + 1) - bj0 + 0.5, np.arange(i0, i1 + 1) - bi0 + 0.5)
    dx, dy = jj - X, ii - Y
    t1 = a[2] * (dx + kap * dy)
    t2 = b[0] * dy
    return float((b[1] - t1 * t1 - t2 * t2).max())


def _check_footprints(dv, pl, tile, off, tx):
    """Each instance's footprint-test byte against a CPU replay from the GPU's
    own record: for every 8x8 footprint of the tile, the 'covers' bit is set
    exactly when the footprint is live and the box covers it, and a footprint
    marked not live holds only exact FP32 zeros of the record (or lies outside
    its box). Returns the numbers of live and culled (instance, footprint)
    pairs inside boxes."""
    keys, recs, fps, boxes = dv["keys"], dv["records"], dv["footprints"], dv["boxes"]
    rec_a, rec_b, rec_c = dv["rec_a"], dv["rec_b"], dv["rec_c"]
    rec_plane = dv["rec_plane"].astype(np.int64)
    fx = tile // 8
    n_live = n_cut = 0
    assert np.all(fps >> (2 * fx * fx) == 0)  # no bits beyond the tile's footprints
    for key, rid, fp in zip(keys.tolist(), recs.tolist(), fps.tolist()):
        p = int(rec_plane[rid])
        local = key - int(off[p])
        ty, txx = divmod(local, int(tx[p]))
        j0, j1 = int(boxes[rid, 0] & 0xFFFF), int(boxes[rid, 0] >> 16)
        i0, i1 = int(boxes[rid, 1] & 0xFFFF), int(boxes[rid, 1] >> 16)
        for f in range(fx * fx):
            fj0, fi0 = txx * tile + (f % fx) * 8, ty * tile + (f // fx) * 8
            live, full = (fp >> (2 * f)) & 1, (fp >> (2 * f + 1)) & 1
            xa, xb, ya, yb = max(fj0, j0), min(fj0 + 7, j1), max(fi0, i0), min(fi0 + 7, i1)
            covers = j0 <= fj0 and j1 >= fj0 + 7 and i0 <= fi0 and i1 >= fi0 + 7
            assert full == (live and covers), (rid, key, f, fp)
            if xa > xb or ya > yb:
                assert not live, (rid, key, f, fp)
                continue
            if live:
                n_live += 1
            else:
                n_cut += 1
                e = _max_exponent(rec_a[rid], rec_b[rid], rec_c[rid], boxes[rid], xa, xb, ya, yb)
                assert e < -126.5, (rid, key, f, e)
    return n_live, n_cut


def _check_tile_lists(r, pl, tile):
    """The GPU's sorted instances against a CPU replay from the GPU's own
    records: for every tile, its records are those whose box meets the tile,
    in ascending record id, minus only pairs whose weights are all exact FP32
    zeros (binning drops those: the record's exact weight exponent is below
    -126.5 at every pixel of the pair); the ranges delimit the tiles; every
    instance's footprint tests hold (see _check_footprints). Returns the
    numbers of kept and dropped (record, tile) pairs."""
    dv = r.debug_views()
    keys, recs, ranges, boxes = dv["keys"], dv["records"], dv["ranges"], dv["boxes"]
    rec_a, rec_b, rec_c = dv["rec_a"], dv["rec_b"], dv["rec_c"]
    rec_plane = dv["rec_plane"].astype(np.int64)
    n_rec = dv["status"]["records"]
    assert len(boxes) == n_rec
    off, tx = _tile_offsets(pl, tile)
    j0s, j1s = boxes[:, 0] & 0xFFFF, boxes[:, 0] >> 16
    i0s, i1s = boxes[:, 1] & 0xFFFF, boxes[:, 1] >> 16
    live = (j0s <= j1s) & (i0s <= i1s)  # empty slots: candidates the exact test rejected
    # sorted order: keys non-decreasing, ascending record id within a tile (stable)
    assert np.all(np.diff(keys.astype(np.int64)) >= 0)
    same = np.diff(keys.astype(np.int64)) == 0
    assert np.all(np.diff(recs.astype(np.int64))[same] > 0)
    got = set(zip(keys.tolist(), recs.tolist()))
    assert len(got) == len(keys)
    kept = dropped = 0
    for rid in np.flatnonzero(live):
        j0, j1, i0, i1 = int(j0s[rid]), int(j1s[rid]), int(i0s[rid]), int(i1s[rid])
        p = int(rec_plane[rid])
        for ty in range(i0 // tile, i1 // tile + 1):
            for txx in range(j0 // tile, j1 // tile + 1):
                key = int(off[p] + ty * tx[p] + txx)
                if (key, int(rid)) in got:
                    got.discard((key, int(rid)))
                    kept += 1
                    continue
                dropped += 1
                e = _max_exponent(rec_a[rid], rec_b[rid], rec_c[rid], boxes[rid], max(j0, txx * tile),
                                  min(j1, txx * tile + tile - 1), max(i0, ty * tile),
                                  min(i1, ty * tile + tile - 1))
                assert e < -126.5, (rid, key, e)  # 2^e underflows to +0 in FP32 (ftz)
    assert not got, f"{len(got)} instances outside their record's box"
    exp_ranges = np.zeros((off[-1], 2), np.uint32)
    for t in range(off[-1]):
        lo = np.searchsorted(keys, t, side="left")
        hi = np.searchsorted(keys, t, side="right")
        if hi > lo:
            exp_ranges[t] = (lo, hi)
    assert np.array_equal(ranges, exp_ranges)
    n_live, n_cut = _check_footprints(dv, pl, tile, off, tx)
    assert n_live > 0
    dv["footprints_live_culled"] = (n_live, n_cut)
    return dv, live, kept, dropped


@pytest.mark.parametrize("tile", [16, 8])
def test_tile_lists_exact(tile):
    rng = np.random.default_rng(21)
    g = synth.gaussians_scale_rot(rng, 2500, 0.02, 0.12)
    pl = synth.planes_random(rng, [(64, 64), (70, 45), (33, 97)])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, tile=tile)
    r, _, _, _ = gpu_render(g, pl, cfg)
    dv, live, kept, dropped = _check_tile_lists(r, pl, tile)
    boxes, rec_plane = dv["boxes"], dv["rec_plane"]
    assert len(boxes) > 100 and kept > 100
    # records and boxes against the oracle's FP64 decisions
    geo = oracle.geometry(g, pl, oracle_config(cfg))
    exp = _expected_records(geo, 2500, len(pl["size"]))
    amb_any = any(_edge_ambiguous(geo, pl, p, gg) for p, gg in exp)
    live_ids = np.flatnonzero(live)
    if not amb_any:
        assert len(exp) == len(live_ids)
        for rid, (p, gg) in zip(live_ids, exp):
            ob = geo["box"][p, gg]
            assert rec_plane[rid] == p
            got = (boxes[rid, 0] & 0xFFFF, boxes[rid, 0] >> 16, boxes[rid, 1] & 0xFFFF,
                   boxes[rid, 1] >> 16)
            assert tuple(int(x) for x in ob) == tuple(int(x) for x in got), (rid, p, gg, ob, got)
    else:  # counts may differ only by ambiguous decisions
        assert abs(len(exp) - len(live_ids)) <= sum(_edge_ambiguous(geo, pl, p, gg) for p, gg in exp)


def test_tile_lists_exact_many_scan_blocks():
    """80 planes (2,048-entry scan blocks then end inside a chunk's run of
    planes) and 6,000 Gaussians: the candidate scan spans 8 blocks and the
    record scan several, their partials added by the cull and the live-tile
    pass; the records are the oracle's visible pairs in (chunk, plane,
    Gaussian) order and the tile lists are exact."""
    rng = np.random.default_rng(25)
    n = 6000
    g = synth.gaussians_scale_rot(rng, n, 0.02, 0.1)
    pl = synth.planes_random(rng, [(24, 24), (20, 31)] * 40)
    P = len(pl["size"])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, tile=16)
    r, _, _, _ = gpu_render(g, pl, cfg)
    assert ((n + 31) // 32) * P > 7 * 2048
    dv, live, kept, dropped = _check_tile_lists(r, pl, 16)
    assert dv["status"]["records"] > 4 * 2048, dv["status"]["records"]
    geo = oracle.geometry(g, pl, oracle_config(cfg))
    exp = _expected_records(geo, n, P)
    E = [(p, tuple(int(x) for x in geo["box"][p, gg])) for p, gg in exp]
    boxes = dv["boxes"].astype(np.int64)
    G = [(int(dv["rec_plane"][rid]), (int(boxes[rid, 0] & 0xFFFF), int(boxes[rid, 0] >> 16),
                                      int(boxes[rid, 1] & 0xFFFF), int(boxes[rid, 1] >> 16)))
         for rid in np.flatnonzero(live)]
    # pairs whose decision may go either way: a box edge within rounding of a
    # pixel boundary, or the plane test within rounding (visible or not)
    amb = sum(_edge_ambiguous(geo, pl, p, gg) for p, gg in exp)
    amb += int((geo["amb_plane"] & ~geo["visible"]).sum())
    # walk both sequences; every difference is one ambiguous pair (a box that
    # differs, a record only one side has)
    i = j = diff = 0
    while i < len(E) and j < len(G):
        if E[i] == G[j]:
            i, j = i + 1, j + 1
        elif E[i][0] == G[j][0] and E[i + 1:i + 3] == G[j + 1:j + 3]:
            i, j, diff = i + 1, j + 1, diff + 1
        elif E[i + 1:i + 2] == G[j:j + 1]:
            i, diff = i + 1, diff + 1
        elif E[i:i + 1] == G[j + 1:j + 2]:
            j, diff = j + 1, diff + 1
        else:
            raise AssertionError(f"records differ at {i} / {j}: {E[i:i + 3]} vs {G[j:j + 3]}")
    diff += (len(E) - i) + (len(G) - j)
    assert diff <= amb, (diff, amb)


def test_tile_lists_thin_gaussians_drop_zero_tiles():
    """Needle- and disc-like Gaussians: their boxes cover many tiles that hold
    only exact zeros; binning drops those (and only those)."""
    rng = np.random.default_rng(23)
    g = synth.gaussians_anisotropic(rng, 3000, ratio_max=1e3)
    pl = synth.planes_random(rng, [(128, 128), (96, 160)])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, tile=16)
    r, _, image, alpha = gpu_render(g, pl, cfg)
    dv, _, kept, dropped = _check_tile_lists(r, pl, 16)
    assert kept > 100 and dropped > 0.1 * kept, (kept, dropped)
    n_live, n_cut = dv["footprints_live_culled"]
    assert n_cut > 0.05 * n_live, (n_live, n_cut)  # footprints of kept tiles culled too


def test_sort_multi_pass_keys():
    """More than 256 tiles: the sort runs two 8-bit passes; order stays exact."""
    rng = np.random.default_rng(22)
    g = synth.gaussians_scale_rot(rng, 4000, 0.01, 0.05)
    pl = synth.planes_random(rng, [(256, 256), (200, 130)])
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, tile=8)
    r, _, _, _ = gpu_render(g, pl, cfg)
    assert r.plan.sort_passes == 2
    dv = r.debug_views()
    keys, recs = dv["keys"].astype(np.int64), dv["records"].astype(np.int64)
    assert np.all(np.diff(keys) >= 0)
    same = np.diff(keys) == 0
    assert np.all(np.diff(recs)[same] > 0)  # stable: ascending record id within a tile


def _grab_u32(r, ptr, count):
    off = ptr - r.ws.data_ptr()
    return r.ws[off:off + 4 * count].view(torch.int32).cpu().numpy().view(np.uint32).copy()


def test_sort_many_tiles_matches_stable_argsort():
    """The radix passes at a size that spans hundreds of sort tiles (each
    tile's digit offsets come from the scan over every earlier tile), and the
    count scans at hundreds of scan blocks (their partials added atomically by
    the cull and the live-tile pass): the sorted (key, record) pairs are exactly
    NumPy's stable sort of the binning's output by tile key, and the ranges
    delimit the tiles."""
    g, pl = synth.workload_aniso_1m(n=200_000)
    g = synth.scale_rot_to_tri(g, 1e-4)
    cfg = R.make_config(cov_param=B.UG_COV_TRI, tile=16)
    params = torch.from_numpy(R.pack_params(g, cfg.cov_param)).cuda()
    r = R.Renderer(len(g["logit"]), pl, cfg)
    r.preprocess(params)  # sizes the workspace
    assert r.plan.sort_passes == 2  # the binning writes the buffers the last pass writes
    kp, vp, rp, bp, *_ = B.ug_debug_views(r.plan, r.ws)
    cap = int(r.plan.instance_capacity)
    for ptr in (kp, vp):  # unwritten instances would read as all ones
        off = ptr - r.ws.data_ptr()
        r.ws[off:off + 4 * cap].fill_(255)
    st = r.preprocess(params)
    n = st["instances"]
    assert n > 300 * 4096, n
    keys0, vals0 = _grab_u32(r, kp, n), _grab_u32(r, vp, n)
    # the binning's output (each record's first instance from the record
    # scan): record slots ascending, each record's tiles ascending, every tile
    # in the box
    tk0 = (keys0 & np.uint32(0x00FFFFFF)).astype(np.int64)
    v0 = vals0.astype(np.int64)
    assert np.all(np.diff(v0) >= 0)
    same_rec = np.diff(v0) == 0
    assert np.all(np.diff(tk0)[same_rec] > 0)
    boxes = _grab_u32(r, bp, 2 * st["records"]).reshape(-1, 2).astype(np.int64)
    rec_plane = _grab_u32(r, B.ug_debug_views(r.plan, r.ws)[7], st["records"]).astype(np.int64)
    off, tx = _tile_offsets(pl, 16)
    local = tk0 - off[rec_plane[v0]]
    ty, txx = local // tx[rec_plane[v0]], local % tx[rec_plane[v0]]
    b = boxes[v0]
    assert np.all(((b[:, 0] & 0xFFFF) >> 4 <= txx) & (txx <= (b[:, 0] >> 16) >> 4))
    assert np.all(((b[:, 1] & 0xFFFF) >> 4 <= ty) & (ty <= (b[:, 1] >> 16) >> 4))
    B.ug_bin_sort(r.plan, r.ws, None)
    assert r.status()["status"] == B.UG_OK
    keys1, vals1 = _grab_u32(r, kp, n), _grab_u32(r, vp, n)
    order = np.argsort(keys0 & np.uint32(0x00FFFFFF), kind="stable")
    assert np.array_equal(keys1, keys0[order])
    assert np.array_equal(vals1, vals0[order])
    ranges = _grab_u32(r, rp, 2 * int(r.plan.total_tiles)).reshape(-1, 2)
    tk = keys1 & np.uint32(0x00FFFFFF)
    t = np.arange(int(r.plan.total_tiles))
    lo, hi = np.searchsorted(tk, t, "left"), np.searchsorted(tk, t, "right")
    exp = np.where((hi > lo)[:, None], np.stack([lo, hi], 1), 0).astype(np.uint32)
    assert np.array_equal(ranges, exp)
    # a second sort of the same instances gives the same bits (deterministic)
    r.preprocess(params)
    B.ug_bin_sort(r.plan, r.ws, None)
    assert np.array_equal(_grab_u32(r, kp, n), keys1)
    assert np.array_equal(_grab_u32(r, vp, n), vals1)


def test_sort_three_passes():
    """More than 65,536 tiles: three 8-bit passes; order and ranges stay exact."""
    rng = np.random.default_rng(24)
    g = synth.gaussians_scale_rot(rng, 60_000, 0.01, 0.05)
    pl = synth.planes_random(rng, [(512, 512)] * 17, origin_range=0.3)
    cfg = R.make_config(cov_param=B.UG_COV_SCALE_ROT, tile=8)
    r, _, _, _ = gpu_render(g, pl, cfg)
    assert r.plan.sort_passes == 3
    dv = r.debug_views()
    keys, recs = dv["keys"].astype(np.int64), dv["records"].astype(np.int64)
    assert len(keys) > 100_000
    assert np.all(np.diff(keys) >= 0)
    same = np.diff(keys) == 0
    assert np.all(np.diff(recs)[same] > 0)
    assert len(set(zip(keys.tolist(), recs.tolist()))) == len(keys)
    t = np.arange(int(r.plan.total_tiles))
    lo, hi = np.searchsorted(keys, t, "left"), np.searchsorted(keys, t, "right")
    exp = np.where((hi > lo)[:, None], np.stack([lo, hi], 1), 0).astype(np.uint32)
    assert np.array_equal(dv["ranges"], exp)
