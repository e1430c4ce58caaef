"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: per-Gaussian records, tile rectangles, sorted keys, values, tile ranges and tile
levels bit-exact; every pixel within 2e-4 absolute per channel of the oracle, or, where the
oracle's margin to the alpha >= 1/255 skip or the T >= 1e-4 stop is below 1e-5, of the
oracle's colour with that decision flipped (such pixels at most 1e-4 per blended
(pixel, Gaussian) pair, plus 3);
live pixels of the foveated render bit-equal to the full render and inherited pixels equal
to their block's top-left pixel.
"""
import numpy as np
import pytest

import oracle
import paper_2507_04147_gb300 as a3fr
from paper_2507_04147_gb300 import synth
import gpu_helpers as gh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def check_eye(r, e, scene_np, cam, tile=16, gaze=None, fv=None, full=False, pixels=None,
              count_frac=0.0):
    n = scene_np.n
    rec, rect, touched, keys, vals = gh.oracle_eye(scene_np, cam, tile)
    assert np.array_equal(r["rec"][e].view(np.uint32), rec.view(np.uint32)), "records differ"
    assert np.array_equal(r["rect"][e].astype(np.int32), rect), "tile rectangles differ"
    n_tiles = oracle.tiles(cam.width, tile) * oracle.tiles(cam.height, tile)
    lo = int(sum(r["stats"]["instances_eye"][:e]))
    hi = lo + int(r["stats"]["instances_eye"][e])
    assert hi - lo == len(keys)
    assert np.array_equal(gh.strip_eye(r["keys"][lo:hi], e, n_tiles), keys), "sorted keys differ"
    assert np.array_equal(r["vals"][lo:hi], vals), "sorted values differ"
    ranges = oracle.tile_ranges(keys, n_tiles)
    gr = r["ranges"][e * n_tiles:(e + 1) * n_tiles].astype(np.int64)
    nonempty = ranges[:, 1] > ranges[:, 0]
    assert np.array_equal(gr[nonempty] - lo, ranges[nonempty].astype(np.int64)), "tile ranges differ"
    assert np.all(gr[~nonempty, 0] == gr[~nonempty, 1])
    if full:
        level = None
        assert np.all(r["levels"][e * n_tiles:(e + 1) * n_tiles] == 4)
    else:
        level = oracle.count_levels(oracle.level_map(cam, tile, fv, gaze), ranges, count_frac)
        assert np.array_equal(r["levels"][e * n_tiles:(e + 1) * n_tiles], level), "levels differ"
    ref = oracle.render(rec, rect, cam, tile, level=level, pixels=pixels)
    img = r["img"][e]
    if pixels is None:
        got = img.reshape(-1, 3)
        info = gh.compare_pixels(got, ref)
        if "t_final" in r:
            ok = ref.margin >= gh.DELTA
            tf = r["t_final"][e].reshape(-1)
            assert np.abs(tf - ref.t_final)[ok].max() <= 2e-4
            nc = r["n_contrib"][e].reshape(-1)
            assert np.array_equal(nc[ok], ref.n_contrib[ok])
            # expected depth: the blend weights (2e-4 each) times depths of a few units
            dz = r["depth"][e].reshape(-1)
            assert np.abs(dz - ref.depth)[ok].max() <= 2e-3
    else:
        got = img[pixels[:, 1], pixels[:, 0]]
        info = gh.compare_pixels(got, ref)
    return info


def fovea_params():
    return oracle.fovea((18.0, 36.0), 0.0, (4, 2, 1)), a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1))


def test_small_single_view_foveated_and_full():
    w = synth.small_single_view()
    cam = w.cameras(0)[0]
    ofv, gfv = fovea_params()
    r = gh.run(w.scene, [cam], gaze=[w.fixed_gaze_px], fovea=gfv)
    assert r["stats"]["status"] == 0
    info = check_eye(r, 0, w.scene, cam, gaze=w.fixed_gaze_px, fv=ofv)
    print("foveated", info)
    rf = gh.run(w.scene, [cam], full=True)
    info = check_eye(rf, 0, w.scene, cam, full=True)
    print("full", info)
    # foveated live pixels are bit-equal to the full render; the rest copy their top-left
    lv = oracle.level_map(cam, 16, ofv, w.fixed_gaze_px)
    ref = oracle.render(*oracle.preprocess(w.scene, cam, 16)[:2], cam, 16, level=lv)
    live = ref.rendered.reshape(256, 256).astype(bool)
    fov, full = r["img"][0], rf["img"][0]
    assert np.array_equal(fov[live], full[live])
    tl = np.repeat(np.repeat(full[0::2, 0::2], 2, axis=0), 2, axis=1)
    assert np.array_equal(fov[~live], tl[~live])


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("binning", [a3fr.BINNING_DIRECT, a3fr.BINNING_SORTED])
def test_stereo_sh3_ragged_image(binning, tile):
    # 200 x 136 leaves partial tiles on the right and bottom edges (at 32-pixel tiles a lane's
    # pixel pair can straddle the image edge)
    scene = synth.uniform_scene(6000, 3, seed=3)
    cams = synth.stereo_cameras(200, 136, yaw_deg=3.0)
    gaze = np.array([[20.0, 120.0], [25.5, 118.25]], np.float32)
    ofv, gfv = fovea_params()
    r = gh.run(scene, cams, gaze=gaze, fovea=gfv, binning=binning, tile=tile)
    assert r["stats"]["status"] == 0 and r["stats"]["n_eyes"] == 2
    for e in range(2):
        print(e, check_eye(r, e, scene, cams[e], tile=tile, gaze=gaze[e], fv=ofv))
    rf = gh.run(scene, cams, full=True, binning=binning, tile=tile)
    for e in range(2):
        print(e, "full", check_eye(rf, e, scene, cams[e], tile=tile, full=True))


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("levels,theta,dtheta", [((4,), (), 0.0), ((4, 1), (18.0,), 2.1),
                                                 ((4, 3, 2, 1), (10.0, 20.0, 35.0), 0.0)])
def test_layer_configurations(levels, theta, dtheta, tile):
    """Every label count a tile can take (the 4-layer case makes 3-label tiles), at both
    tilings: with 32-pixel tiles each count is its own instantiation of the composite."""
    scene = synth.uniform_scene(4000, 1, seed=5)
    cam = synth.pinhole_camera(160, 144, 90.0, -2.0)
    gaze = (101.3, 40.7)
    ofv = oracle.fovea(theta, dtheta, levels)
    gfv = a3fr.Fovea(theta, dtheta, levels)
    r = gh.run(scene, [cam], gaze=[gaze], fovea=gfv, tile=tile)
    print(check_eye(r, 0, scene, cam, tile=tile, gaze=gaze, fv=ofv))
    n_tiles = oracle.tiles(160, tile) * oracle.tiles(144, tile)
    assert set(levels) <= set(r["levels"][:n_tiles].tolist()) | {1}


@pytest.mark.parametrize("tile", [16, 32])
def test_degenerate_scenes(tile):
    cam = synth.pinhole_camera(64, 48)
    # no Gaussians (foveated and full: every tile is an empty work item)
    empty = synth.uniform_scene(0, 0, seed=1)
    r = gh.run(empty, [cam], full=True, tile=tile)
    assert r["stats"]["instances"] == 0 and np.all(r["img"] == 0)
    r = gh.run(empty, [cam], gaze=[(20.0, 20.0)], fovea=a3fr.Fovea(), tile=tile)
    assert r["stats"]["instances"] == 0 and np.all(r["img"] == 0)
    # one Gaussian, visible; one behind the camera
    one = synth.uniform_scene(1, 0, seed=2)
    r = gh.run(one, [cam], full=True, tile=tile)
    check_eye(r, 0, one, cam, tile=tile, full=True)
    behind = synth.uniform_scene(1, 0, seed=2)
    behind.means[:, 2] = -3.0
    r = gh.run(behind, [cam], full=True, tile=tile)
    assert r["stats"]["instances"] == 0 and np.all(r["img"] == 0)
    # a huge Gaussian covering every tile in front of small ones
    s = synth.uniform_scene(500, 2, seed=4)
    s.means[0] = [0.0, 0.0, 2.05]
    s.log_scales[0] = [0.5, 0.5, 0.5]
    r = gh.run(s, [cam], gaze=[(0.0, 0.0)], fovea=a3fr.Fovea(), tile=tile)
    check_eye(r, 0, s, cam, tile=tile, gaze=(0.0, 0.0), fv=oracle.fovea())
    assert r["rect"][0, 0].tolist() == [0, 0, oracle.tiles(64, tile), oracle.tiles(48, tile)]


@pytest.mark.parametrize("binning", [a3fr.BINNING_DIRECT, a3fr.BINNING_SORTED])
def test_depth_range_wider_than_the_rebase(binning):
    # depths 0.5 .. 40: the visible depth keys span more than 2^24, so they are not rebased
    # and the top 8-bit digit differs between near and far Gaussians; the last depth pass
    # then really permutes (the other parity scenes, all at depths 2 .. 6, take the
    # identity last pass that writes nothing)
    s = synth.uniform_scene(3000, 1, seed=21)
    z = np.float32(0.5) * np.exp(np.linspace(0.0, np.log(80.0), s.n)).astype(np.float32)
    np.random.Generator(np.random.PCG64(22)).shuffle(z)
    s.means[:, 2] = z
    s.means[:, 0] *= 0.8 * z
    s.means[:, 1] *= 0.5 * z
    key = z.view(np.uint32)
    assert int(key.max()) - int(key.min()) >= 1 << 24 and (key.max() >> 24) != (key.min() >> 24)
    cam = synth.pinhole_camera(96, 64)
    fv, fa = fovea_params()
    for full in (True, False):
        r = gh.run(s, [cam], gaze=None if full else [(40.0, 30.0)], fovea=None if full else fa,
                   full=full, binning=binning)
        assert r["stats"]["status"] == 0
        check_eye(r, 0, s, cam, full=full, gaze=(40.0, 30.0), fv=fv)


@pytest.mark.parametrize("tile", [16, 32])
def test_sorted_binning_of_single_tile_gaussians(tile):
    # tiny Gaussians cover one tile (a few near tile borders two or four) and some lie behind
    # the camera: the tile sort's first pass then sees a partition's 4,096 instance slots
    # spread over more entries than it stages at once (several windows per partition), and
    # entries without instances at the end of the depth order
    s = synth.uniform_scene(24000, 0, seed=31, log_scale_mean=-9.0)
    s.means[::7, 2] = -s.means[::7, 2]
    cam = synth.pinhole_camera(256, 256)
    rec, rect, touched, keys, vals = gh.oracle_eye(s, cam, tile)
    vis = touched > 0
    assert (~vis).sum() > 1000 and len(keys) < 2 * vis.sum()
    fv, fa = fovea_params()
    for full in (True, False):
        r = gh.run(s, [cam], gaze=None if full else [(100.0, 150.0)], fovea=None if full else fa,
                   full=full, binning=a3fr.BINNING_SORTED, tile=tile)
        assert r["stats"]["status"] == 0
        check_eye(r, 0, s, cam, tile=tile, full=full, gaze=(100.0, 150.0), fv=fv)


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("binning", [a3fr.BINNING_DIRECT, a3fr.BINNING_SORTED])
def test_capacity_overflow_sets_status_without_fault(binning, tile):
    w = synth.small_single_view()
    cam = w.cameras(0)[0]
    for full in (True, False):
        r = gh.run(w.scene, [cam], full=full, gaze=[w.fixed_gaze_px], fovea=a3fr.Fovea(),
                   capacity=1000, binning=binning, tile=tile)
        st = r["stats"]
        assert st["status"] & a3fr.STATUS_CAPACITY
        assert st["instances"] == 1000 and st["capacity"] == 1000
        assert np.isfinite(r["img"]).all()


def test_repeated_renders_are_deterministic_and_counters_accumulate():
    import torch
    w = synth.small_single_view()
    cam = w.cameras(0)[0]
    s = a3fr.Scene.from_numpy(w.scene)
    s.set_camera(0, cam)
    s.set_gaze([w.fixed_gaze_px])
    s.keep_aux(True)   # evaluations and blends are counted with the auxiliary outputs
    a = s.render_foveated().clone()
    s.stats(reset=True)
    for _ in range(3):
        b = s.render_foveated()
    st = s.stats()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert st["renders"] == 3 and st["evaluations"] > 0 and st["status"] == 0
    assert 0 < st["contributions"] <= st["evaluations"]


@pytest.mark.parametrize("tile,binning,full", [(16, a3fr.BINNING_SORTED, False), (32, a3fr.BINNING_DIRECT, False),
                                              (16, a3fr.BINNING_DIRECT, False), (32, a3fr.BINNING_DIRECT, True)])
def test_stereo_500k_sh3_sampled_pixels(tile, binning, full):
    """The benchmark workload at full size: records and keys in full, pixels sampled, under
    both binning paths (16-pixel tiles: 12,800 tiles, 4 bands per chunk in the direct path),
    and the benchmark's configuration (32-pixel tiles, direct binning) also at full
    resolution."""
    w = synth.stereo_500k(frames=240)
    traj = synth.gaze_trajectory(240)
    frame = 137
    cams = w.cameras(frame)
    gaze = w.gaze(frame, traj)
    ofv, gfv = fovea_params()
    r = gh.run(w.scene, cams, gaze=gaze, fovea=gfv, keep_aux=False, tile=tile, binning=binning, full=full)
    assert r["stats"]["status"] == 0
    rng = np.random.default_rng(frame)
    for e in range(2):
        pix = np.stack([rng.integers(0, 1280, 1500), rng.integers(0, 1280, 1500)], axis=1)
        # plus every pixel of the tile row through the gaze (crosses all three layers)
        gy = int(np.clip(gaze[e][1], 0, 1279)) // tile * tile
        band = np.stack(np.meshgrid(np.arange(0, 1280, 3), np.arange(gy, gy + tile, 5)), -1).reshape(-1, 2)
        pix = np.concatenate([pix, band]).astype(np.int32)
        print(e, check_eye(r, e, w.scene, cams[e], tile=tile, gaze=gaze[e], fv=ofv, pixels=pix, full=full))


@pytest.mark.parametrize("tile,full,batch_mult", [(32, False, 1), (16, False, 1), (32, True, 1), (32, False, 2)])
def test_stereo_3m_clustered_full_size(tile, full, batch_mult):
    """The 3M-Gaussian clustered stereo 2064x2208 frame at full size, foveated (and at full
    resolution with 32-pixel tiles; and with the staging batch the autotuner picks for this
    workload, 32-pixel tiles x 2), in the binning the library picks there (sort-based: 8,970 tiles at 32 pixels, 35,604 at 16):
    records, rectangles, every sorted key and value (about 22M and 50M instances per
    frame) and the tile ranges of both eyes bit-exact; pixels within the parity bar on a
    random sample, on the tile row through the gaze (all three layers) and on every pixel
    of the heaviest tiles (the longest lists, with Beta(0.5, 0.5) opacities near the 0.99
    clamp and the early stop)."""
    w = synth.stereo_3m_clustered(frames=240)
    traj = synth.gaze_trajectory(240)
    frame = 97
    cams = w.cameras(frame)
    gaze = w.gaze(frame, traj)
    ofv, gfv = fovea_params()
    r = gh.run(w.scene, cams, gaze=gaze, fovea=gfv, keep_aux=False, tile=tile, full=full,
               batch_mult=batch_mult)
    assert r["stats"]["status"] == 0
    W, H = cams[0].width, cams[0].height
    tx, ty = oracle.tiles(W, tile), oracle.tiles(H, tile)
    n_tiles = tx * ty
    rng = np.random.default_rng(frame + tile)
    heavy_per_eye = 4 if tile == 32 else 8
    for e in range(2):
        pix = [np.stack([rng.integers(0, W, 1000), rng.integers(0, H, 1000)], axis=1)]
        gy = int(np.clip(gaze[e][1], 0, H - 1)) // tile * tile
        pix.append(np.stack(np.meshgrid(np.arange(0, W, 7), np.arange(gy, min(gy + tile, H), 4)),
                            -1).reshape(-1, 2))
        cnt = r["ranges"][e * n_tiles:(e + 1) * n_tiles].astype(np.int64)
        cnt = cnt[:, 1] - cnt[:, 0]
        for t in np.argsort(-cnt, kind="stable")[:heavy_per_eye]:
            x0, y0 = (t % tx) * tile, (t // tx) * tile
            xs, ys = np.meshgrid(np.arange(x0, min(x0 + tile, W)), np.arange(y0, min(y0 + tile, H)))
            pix.append(np.stack([xs.reshape(-1), ys.reshape(-1)], axis=1))
        pix = np.concatenate(pix).astype(np.int32)
        print(e, "heaviest tile instances", int(cnt.max()),
              check_eye(r, e, w.scene, cams[e], tile=tile, gaze=gaze[e], fv=ofv, pixels=pix,
                        full=full))
    r["scene"].close()


@pytest.mark.parametrize("tile", [16, 32])
def test_graph_mode_matches_direct_launches_bitwise(tile):
    """Replayed CUDA graphs see each render's cameras, gaze and output through device-resident
    parameters, so they must reproduce the directly launched renders exactly (with 32-pixel
    tiles the composite is one persistent launch taking work items from a device counter)."""
    import torch
    w = synth.stereo_500k(frames=240)
    scene_np = w.scene.subset(np.arange(60000))
    traj = synth.gaze_trajectory(240)
    direct = a3fr.Scene.from_numpy(scene_np, tile=tile)
    graph = a3fr.Scene.from_numpy(scene_np, tile=tile)
    graph.graph_mode(True)
    for s in (direct, graph):
        for e, c in enumerate(w.cameras(0)):
            s.set_camera(e, c)
    outs = {}
    for name, s in (("direct", direct), ("graph", graph)):
        imgs = []
        for f in (0, 7, 50, 51, 130):
            for e, c in enumerate(w.cameras(f)):
                s.set_camera(e, c)
            s.set_gaze(w.gaze(f, traj))
            imgs.append(s.render_foveated(a3fr.Fovea()).clone())
            imgs.append(s.render_full().clone())
        torch.cuda.synchronize()
        outs[name] = imgs
    for a, b in zip(outs["direct"], outs["graph"]):
        assert torch.equal(a, b)
    st = graph.stats()
    assert st["status"] == 0


def test_stage_timing_in_graph_mode():
    """With stage timing on, a graph-mode render is timed around its two graphs (precompute,
    composite) and renders the same images as untimed graph renders."""
    import torch
    w = synth.stereo_500k(frames=240)
    scene_np = w.scene.subset(np.arange(40000))
    traj = synth.gaze_trajectory(240)
    imgs = {}
    for timed in (False, True):
        s = a3fr.Scene.from_numpy(scene_np, tile=32)
        s.graph_mode(True)
        out = []
        for f in (0, 3, 0, 9, 20):
            for e, c in enumerate(w.cameras(f)):
                s.set_camera(e, c)
            s.set_gaze(w.gaze(f, traj))
            if timed and len(out) == 2:
                s.stage_timing(8)   # after the graphs were captured untimed
            out.append(s.render_foveated(a3fr.Fovea()).clone())
        torch.cuda.synchronize()
        imgs[timed] = out
        if timed:
            st = s.stage_times(8)
            assert st.shape == (3, 5)
            assert np.all(st[:, 0] > 0.0) and np.all(st[:, 4] > 0.0)
            assert np.all(st[:, 1:4] < 0.05 * st[:, 4])
            s.stage_timing(0)
        assert s.stats()["status"] == 0
        s.close()
    for a, b in zip(imgs[False], imgs[True]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("batch_mult", [1, 2])
def test_tile32_foveated_and_full(batch_mult):
    """32-pixel tiles (one CTA per tile rendering all its labels) against the oracle run with
    32-pixel tiles."""
    scene = synth.uniform_scene(8000, 3, seed=13)
    cams = synth.stereo_cameras(200, 136, yaw_deg=2.0)
    gaze = np.array([[70.0, 60.0], [66.0, 61.0]], np.float32)
    ofv, gfv = fovea_params()
    r = gh.run(scene, cams, gaze=gaze, fovea=gfv, tile=32, batch_mult=batch_mult)
    assert r["stats"]["status"] == 0
    for e in range(2):
        print(e, check_eye(r, e, scene, cams[e], tile=32, gaze=gaze[e], fv=ofv))
    rf = gh.run(scene, cams, full=True, tile=32, batch_mult=batch_mult)
    for e in range(2):
        check_eye(rf, e, scene, cams[e], tile=32, full=True)


def test_batch_multiplier_renders_bitwise_equal():
    """Staging two Gaussians per thread changes only the batching, not any pixel's sequence."""
    w = synth.small_single_view()
    cam = w.cameras(0)[0]
    for tile in (16, 32):
        a = gh.run(w.scene, [cam], gaze=[w.fixed_gaze_px], fovea=a3fr.Fovea(), tile=tile, batch_mult=1)
        b = gh.run(w.scene, [cam], gaze=[w.fixed_gaze_px], fovea=a3fr.Fovea(), tile=tile, batch_mult=2)
        assert np.array_equal(a["img"], b["img"])


def test_autotune_picks_a_configuration_and_renders_it():
    import torch
    w = synth.stereo_500k(frames=240)
    scene_np = w.scene.subset(np.arange(100000))
    cams = synth.stereo_cameras(640, 640, yaw_deg=1.0)
    s = a3fr.Scene.from_numpy(scene_np)
    for e, c in enumerate(cams):
        s.set_camera(e, c)
    s.set_gaze([[300.0, 330.0], [290.0, 330.0]])
    res = s.autotune(a3fr.Fovea(), timed_renders=3)
    print(res)
    assert res["tile"] in (16, 32) and res["batch_mult"] in (1, 2)
    assert all(v > 0 for v in res["ms"].values())
    assert res["ms"][(res["tile"], res["batch_mult"])] == min(res["ms"].values())
    img = s.render_foveated(a3fr.Fovea()).clone()
    s.set_tile(16)
    s.set_batch(1)
    ref = s.render_foveated(a3fr.Fovea())
    torch.cuda.synchronize()
    if res["tile"] == 16:
        assert torch.equal(img, ref)
    s.close()


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("width,height", [(200, 136), (201, 137)])
def test_interpolating_fill(tile, width, height):
    """Skipped pixels interpolated from rendered neighbours: bit-equal to the oracle's rule
    applied to the GPU's rendered pixels, rendered pixels unchanged, and within the pixel
    tolerance of the oracle's own filled image.  Odd sizes cut the last blocks."""
    scene = synth.uniform_scene(6000, 3, seed=3)
    cams = synth.stereo_cameras(width, height, yaw_deg=3.0)
    gaze = np.array([[60.0, 70.0], [58.5, 70.0]], np.float32)
    ofv = oracle.fovea((18.0, 36.0), 0.0, (4, 2, 1))
    inh = gh.run(scene, cams, gaze=gaze, fovea=a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1)), tile=tile)
    itp = gh.run(scene, cams, gaze=gaze, tile=tile,
                 fovea=a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1), fill=a3fr.FILL_INTERPOLATE))
    for e in range(2):
        lv = oracle.level_map(cams[e], tile, ofv, gaze[e])
        ref = oracle.render(*oracle.preprocess(scene, cams[e], tile)[:2], cams[e], tile, level=lv)
        live = ref.rendered.reshape(height, width).astype(bool)
        assert np.array_equal(itp["img"][e][live], inh["img"][e][live])
        exact = oracle.fill_interpolate(inh["img"][e], live)
        assert np.array_equal(itp["img"][e], exact)
        # the oracle's rendered pixels, each taken as the oracle's colour or -- where the
        # GPU took a near-threshold decision the other way -- its flipped-decision colour,
        # then filled by the oracle's rule: every pixel within the tolerance
        gh.compare_pixels(inh["img"][e].reshape(-1, 3), ref)
        g = inh["img"][e].reshape(-1, 3).astype(np.float64)
        alt = ((ref.margin < gh.DELTA) & (np.abs(g - ref.rgb_alt).max(1) < np.abs(g - ref.rgb).max(1)))
        chosen = np.where(alt[:, None], ref.rgb_alt, ref.rgb).reshape(height, width, 3)
        filled_ref = oracle.fill_interpolate(chosen, live)
        assert np.abs(itp["img"][e] - filled_ref).max() <= gh.TOL


def test_interpolating_fill_3m_full_size_sampled():
    """The interpolating fill on the 3M clustered stereo 2064x2208 frame (32-pixel tiles):
    every rendered pixel unchanged, and sampled skipped pixels -- random ones plus every pixel
    of the tile row through the gaze and of the tile boundaries it crosses -- bit-equal to the
    oracle's rule applied to the pixel's neighbourhood in the inherit render (a window of
    3x3 pixels cut at the image edge, as the image cuts the rule)."""
    import torch
    w = synth.stereo_3m_clustered(frames=240)
    traj = synth.gaze_trajectory(240)
    frame = 97
    cams = w.cameras(frame)
    gaze = w.gaze(frame, traj)
    ofv, gfv = fovea_params()
    tile = 32
    s = a3fr.Scene.from_numpy(w.scene, tile=tile)
    for e, c in enumerate(cams):
        s.set_camera(e, c)
    s.set_gaze(gaze)
    inh = s.render_foveated(gfv).clone()
    itp = s.render_foveated(a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1), fill=a3fr.FILL_INTERPOLATE)).clone()
    st = s.stats()
    torch.cuda.synchronize()
    s.close()
    assert st["status"] == 0
    inh, itp = inh.cpu().numpy(), itp.cpu().numpy()
    W, H = cams[0].width, cams[0].height
    ys, xs = np.mgrid[0:H, 0:W]
    label = np.where((xs & 1) == (ys & 1), np.where(xs & 1, 1, 0), np.where(xs & 1, 2, 3))
    rng = np.random.default_rng(frame)
    for e in range(2):
        lv = oracle.level_map(cams[e], tile, ofv, gaze[e]).reshape(oracle.tiles(H, tile), oracle.tiles(W, tile))
        live = label < lv[ys // tile, xs // tile]
        assert (~live).any() and live.any()
        assert np.array_equal(itp[e][live], inh[e][live])
        skipped = np.argwhere(~live)                                   # (y, x)
        pick = [skipped[rng.choice(len(skipped), 3000, replace=False)]]
        gy = int(np.clip(gaze[e][1], 0, H - 1)) // tile * tile
        row = skipped[(skipped[:, 0] >= gy) & (skipped[:, 0] < gy + tile)]
        pick.append(row[::3])
        edge = skipped[((skipped[:, 1] % tile) == 0) | ((skipped[:, 1] % tile) == tile - 1) |
                       ((skipped[:, 0] % tile) == 0) | ((skipped[:, 0] % tile) == tile - 1)]
        pick.append(edge[rng.choice(len(edge), 2000, replace=False)])
        pick.append(np.array([[H - 1, W - 1], [H - 1, 0], [0, W - 1]]))
        bad = 0
        for y, x in np.concatenate(pick):
            if live[y, x]:
                continue
            y0, y1, x0, x1 = max(y - 1, 0), min(y + 2, H), max(x - 1, 0), min(x + 2, W)
            want = oracle.fill_interpolate(inh[e][y0:y1, x0:x1], live[y0:y1, x0:x1])[y - y0, x - x0]
            bad += int(not np.array_equal(itp[e][y, x], want))
        assert bad == 0, (e, bad)


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("count_frac", [0.2, 1.0])
def test_count_based_tile_levels(tile, count_frac):
    """Tile levels by Gaussian count: levels bit-equal to the oracle's rule over the oracle's
    own tile ranges, pixels within the parity bar; the rule changes some tiles, and the
    scene's cached graphs keep count-based and plain renders apart."""
    import torch
    scene = synth.uniform_scene(6000, 3, seed=3)
    cams = synth.stereo_cameras(200, 136, yaw_deg=3.0)
    gaze = np.array([[60.0, 70.0], [58.5, 70.0]], np.float32)
    ofv = oracle.fovea((18.0, 36.0), 0.0, (4, 3, 2))
    gfv = a3fr.Fovea((18.0, 36.0), 0.0, (4, 3, 2), count_frac=count_frac)
    r = gh.run(scene, cams, gaze=gaze, fovea=gfv, tile=tile)
    assert r["stats"]["status"] == 0
    n_tiles = oracle.tiles(200, tile) * oracle.tiles(136, tile)
    changed = 0
    for e in range(2):
        print(e, check_eye(r, e, scene, cams[e], tile=tile, gaze=gaze[e], fv=ofv, count_frac=count_frac))
        plain = oracle.level_map(cams[e], tile, ofv, gaze[e])
        changed += int((r["levels"][e * n_tiles:(e + 1) * n_tiles] != plain).sum())
    assert changed > 0
    s = r["scene"]
    for frac in (0.0, count_frac, 0.0):
        s.render_foveated(a3fr.Fovea((18.0, 36.0), 0.0, (4, 3, 2), count_frac=frac))
        torch.cuda.synchronize()
        lv = s.buffer(a3fr.BUF_LEVELS, torch.uint8).cpu().numpy()
        assert np.array_equal(lv, r["levels"]) == (frac == count_frac)
    s.close()
