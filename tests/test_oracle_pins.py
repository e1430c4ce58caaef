"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test is chosen so that a plausible slip in the oracle -- a dropped term, a wrong
sign or index, a transposed operand, a wrong threshold -- fails at least one of them:

* closed forms: on-axis isotropic Gaussian (EWA covariance, conic, radius, pixel values);
* library routines: scipy rotations (quaternion convention and R diag(s^2) R^T),
  scipy real spherical harmonics (SH constants and index map), finite differences
  of the pinhole projection (Jacobian signs and indices), libm exp (the project exp);
* invariants: weight sum / white colour, input-order invariance, foveated live pixels
  equal to the full render, inherited pixels equal to their block's top-left;
* brute force: fp64 per-pixel compositing on tiny scenes, brute-force tile membership
  and Python sorting for the keys, brute-force geometry for the level map.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2507_04147_gb300 import synth
import brute_fp64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _one_gaussian(mean, log_scale, quat=(1, 0, 0, 0), logit=2.0, colour=(0.7, 0.4, 0.2)):
    s = synth.Scene(np.array([mean], np.float32), np.array([log_scale], np.float32),
                    np.array([quat], np.float32), np.array([logit], np.float32),
                    np.zeros((1, 1, 3), np.float32), 0)
    s.sh[0, 0, :] = (np.array(colour) - 0.5) / (0.5 / math.sqrt(math.pi))
    return s


def _cam(width=64, height=64, yaw=0.0, offset=0.0):
    return synth.pinhole_camera(width, height, 90.0, yaw, offset)


# ------------------------------------------------------------------ exp
def test_project_exp_accuracy():
    xs = np.concatenate([np.linspace(-87, 88, 20001), np.random.default_rng(3).normal(-4, 2, 5000)])
    worst = 0.0
    for x in xs.astype(np.float32):
        ref = math.exp(float(x))
        got = oracle.exp32(float(x))
        worst = max(worst, abs(got - ref) / ref)
    assert worst < 2.0 ** -21, worst          # within a few fp32 ulp of the true exp
    assert oracle.exp32(0.0) == 1.0


# ------------------------------------------------------------------ SH
def test_sh_basis_matches_scipy_real_harmonics():
    rng = np.random.default_rng(0)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ours = np.array([oracle.sh_basis(x, 3) for x in d.astype(np.float32)], dtype=np.float64)
    for l in range(4):
        for m in range(-l, l + 1):
            k = l * l + l + m
            ref = brute_fp64.real_sh(l, m, d)
            # same function up to one sign per coefficient, and that sign is (-1)^m
            np.testing.assert_allclose(ours[:, k], (-1) ** m * ref, atol=2e-6)


def test_sh_degree0_colour_equals_drawn_base_colour():
    scene = synth.uniform_scene(500, 0, seed=4)
    cam = _cam()
    rec, rect, touched = oracle.preprocess(scene, cam, 16)
    rng = np.random.Generator(np.random.PCG64(4))
    rng.uniform(-1, 1, size=(500, 3)); rng.normal(size=(500, 3)); rng.normal(size=(500, 4))
    rng.normal(size=500)
    base = rng.uniform(0, 1, size=(500, 3))
    vis = rec[:, 11] > 0
    np.testing.assert_allclose(rec[vis, 6:9], base[vis], atol=2e-6)


# ------------------------------------------------------------------ projection
def test_on_axis_isotropic_closed_form():
    """Isotropic Gaussian on the optical axis: Sigma' = ((f S / z)^2 + 0.3) I."""
    z, ls = 3.0, -3.0
    cam = _cam(64, 64)
    scene = _one_gaussian((0.0, 0.0, z), (ls, ls, ls))
    rec, rect, touched = oracle.preprocess(scene, cam, 16)
    s2 = (cam.fx * math.exp(ls) / z) ** 2 + 0.3
    assert rec[0, 11] == 1.0
    np.testing.assert_allclose(rec[0, 0:2], [cam.cx, cam.cy], atol=1e-5)
    np.testing.assert_allclose(rec[0, 2:5], [1 / s2, 0.0, 1 / s2], rtol=1e-5, atol=1e-7)
    lam = 0.5 * (2 * s2) + math.sqrt(0.1)           # the eigenvalue floor applies: disc = 0
    assert rec[0, 10] == math.ceil(3 * math.sqrt(lam))
    np.testing.assert_allclose(rec[0, 5], 1 / (1 + math.exp(-2.0)), rtol=1e-6)
    np.testing.assert_allclose(rec[0, 9], z, rtol=1e-7)


@pytest.mark.parametrize("yaw", [0.0, 23.0])
def test_covariance_matches_scipy_rotation_on_axis(yaw):
    """Recover Sigma_cam[:2,:2] from the conic and compare with scipy's rotation."""
    rng = np.random.default_rng(7)
    cam = _cam(256, 256, yaw=yaw)
    Rc = cam.world_to_cam[:, :3].astype(np.float64)
    z = 3.5
    mean = Rc.T @ np.array([0.0, 0.0, z])              # on the optical axis
    for _ in range(20):
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        ls = rng.normal(-3.0, 0.5, size=3)
        scene = _one_gaussian(mean, ls, q)
        rec, _, _ = oracle.preprocess(scene, cam, 16)
        a, b, c = rec[0, 2], rec[0, 3], rec[0, 4]
        cov2 = np.linalg.inv(np.array([[a, b], [b, c]], np.float64)) - 0.3 * np.eye(2)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        sigma = R @ np.diag(np.exp(2 * ls)) @ R.T
        cam_sigma = Rc @ sigma @ Rc.T
        ref = (cam.fx / z) ** 2 * cam_sigma[:2, :2]
        np.testing.assert_allclose(cov2, ref, rtol=2e-3, atol=2e-3 * np.abs(ref).max())


def test_covariance_eigenvalues_are_exp_2s():
    cam = _cam(256, 256)
    rng = np.random.default_rng(11)
    for _ in range(10):
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        ls = rng.normal(-2.5, 0.4, size=3)
        # on the optical axis of an identity camera the projected covariance is the
        # top-left 2x2 block of R diag(exp(2 s)) R^T scaled by (f / z)^2
        scene = _one_gaussian((0, 0, 3.0), ls, q)
        rec, _, _ = oracle.preprocess(scene, cam, 16)
        cov2 = np.linalg.inv(np.array([[rec[0, 2], rec[0, 3]], [rec[0, 3], rec[0, 4]]], np.float64)) - 0.3 * np.eye(2)
        cov2 /= (cam.fx / 3.0) ** 2
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        full = R @ np.diag(np.exp(2 * ls)) @ R.T
        np.testing.assert_allclose(np.linalg.eigvalsh(full), np.sort(np.exp(2 * ls)), rtol=1e-9)
        np.testing.assert_allclose(cov2, full[:2, :2], rtol=2e-3, atol=1e-3 * np.exp(2 * ls).max())


def test_jacobian_matches_finite_differences_off_axis():
    """Off-axis Gaussian: Sigma' = J Sigma J^T + 0.3 I with J from central differences."""
    cam = _cam(256, 256, yaw=10.0)
    Rc = cam.world_to_cam[:, :3].astype(np.float64)
    tc = cam.world_to_cam[:, 3].astype(np.float64)
    rng = np.random.default_rng(5)

    def proj(t):
        return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])

    for _ in range(20):
        tcam = np.array([rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), rng.uniform(2, 5)])
        mean = Rc.T @ (tcam - tc)
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        ls = rng.normal(-3.0, 0.3, size=3)
        scene = _one_gaussian(mean, ls, q)
        rec, _, _ = oracle.preprocess(scene, cam, 16)
        h = 1e-5
        J = np.zeros((2, 3))
        for j in range(3):
            e = np.zeros(3); e[j] = h
            J[:, j] = (proj(tcam + e) - proj(tcam - e)) / (2 * h)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        sigma = Rc @ R @ np.diag(np.exp(2 * ls)) @ R.T @ Rc.T
        ref = J @ sigma @ J.T + 0.3 * np.eye(2)
        got = np.linalg.inv(np.array([[rec[0, 2], rec[0, 3]], [rec[0, 3], rec[0, 4]]], np.float64))
        np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
        np.testing.assert_allclose(rec[0, 0:2], proj(tcam), atol=2e-4)


def test_jacobian_clamp_far_off_screen():
    """Beyond 1.3 tan(fov/2) the Jacobian is evaluated at the clamped point."""
    cam = _cam(64, 64)
    tcam = np.array([3.0, 0.0, 1.0])          # tx/tz = 3 > 1.3 * 0.5 * 64 / 32 = 1.3
    ls = (-1.0, -1.0, -1.0)
    scene = _one_gaussian(tcam, ls)
    rec, rect, _ = oracle.preprocess(scene, cam, 16)
    s = math.exp(-1.0)
    xc = 1.3 * tcam[2]
    J = np.array([[cam.fx / tcam[2], 0, -cam.fx * xc / tcam[2] ** 2], [0, cam.fy / tcam[2], 0]])
    ref = J @ (s * s * np.eye(3)) @ J.T + 0.3 * np.eye(2)
    if rec[0, 11]:
        got = np.linalg.inv(np.array([[rec[0, 2], rec[0, 3]], [rec[0, 3], rec[0, 4]]], np.float64))
        np.testing.assert_allclose(got, ref, rtol=1e-4)
    else:   # entirely off the image: must then have no tiles
        assert rect[0].tolist() == [0, 0, 0, 0]


def test_near_plane_and_offscreen_culling():
    cam = _cam(64, 64)
    behind = _one_gaussian((0, 0, 0.1), (-3, -3, -3))
    rec, rect, touched = oracle.preprocess(behind, cam, 16)
    assert rec[0, 11] == 0 and touched[0] == 0
    far = _one_gaussian((50.0, 0, 2.0), (-3, -3, -3))
    rec, rect, touched = oracle.preprocess(far, cam, 16)
    assert touched[0] == 0


# ------------------------------------------------------------------ compositing
@pytest.mark.parametrize("logit", [1.0, 6.0])     # 6.0: opacity 0.9975 hits the 0.99 clamp
def test_single_gaussian_pixels_closed_form(logit):
    z, ls = 2.5, -3.2
    colour = np.array([0.7, 0.4, 0.2])
    cam = _cam(64, 64)
    scene = _one_gaussian((0.0, 0.0, z), (ls, ls, ls), logit=logit, colour=colour)
    rec, rect, _ = oracle.preprocess(scene, cam, 16)
    img = oracle.render(rec, rect, cam, 16)
    rgb = img.rgb.reshape(64, 64, 3)
    s2 = (cam.fx * math.exp(ls) / z) ** 2 + 0.3
    op = 1 / (1 + math.exp(-logit))
    x0, y0, x1, y1 = rect[0]
    worst = 0.0
    for y in range(64):
        for x in range(64):
            inside = x0 <= x // 16 < x1 and y0 <= y // 16 < y1
            d2 = (x - cam.cx) ** 2 + (y - cam.cy) ** 2
            a = min(0.99, op * math.exp(-0.5 * d2 / s2))
            ref = colour * a if (inside and a >= 1 / 255) else np.zeros(3)
            if img.margin[y * 64 + x] < 1e-4:
                continue
            worst = max(worst, np.abs(rgb[y, x] - ref).max())
    assert worst < 2e-6


def test_stack_front_to_back_and_early_stop_closed_form():
    """Five coincident-centre Gaussians of opacity 0.95 at increasing depth: the centre
    pixel blends the three nearest front to back, then T would fall to 6.25e-6 < 1e-4."""
    colours = np.array([[0.9, 0.1, 0.1], [0.1, 0.8, 0.1], [0.1, 0.1, 0.7], [0.5, 0.5, 0.5], [0.3, 0.6, 0.9]])
    depths = [2.0, 2.4, 2.8, 3.2, 3.6]
    logit = math.log(0.95 / 0.05)
    order = [3, 0, 4, 2, 1]                     # input order differs from depth order
    scene = synth.Scene(np.array([[0, 0, depths[k]] for k in order], np.float32),
                        np.full((5, 3), -3.0, np.float32), np.tile(np.float32([1, 0, 0, 0]), (5, 1)),
                        np.full(5, logit, np.float32), np.zeros((5, 1, 3), np.float32), 0)
    scene.sh[:, 0, :] = (colours[order] - 0.5) / (0.5 / math.sqrt(math.pi))
    cam = synth.pinhole_camera(33, 33)          # principal point (16, 16) is a pixel centre
    rec, rect, _ = oracle.preprocess(scene, cam, 16)
    img = oracle.render(rec, rect, cam, 16)
    p = 16 * 33 + 16
    ref = sum(colours[k] * 0.95 * 0.05 ** k for k in range(3))
    np.testing.assert_allclose(img.rgb[p], ref, rtol=1e-5)
    np.testing.assert_allclose(img.t_final[p], 0.05 ** 3, rtol=1e-4)
    assert img.n_contrib[p] == 3 and img.n_eval[p] == 4 and img.n_blend[p] == 3
    # expected depth: the same blend weights applied to the three depths
    np.testing.assert_allclose(img.depth[p], sum(depths[k] * 0.95 * 0.05 ** k for k in range(3)),
                               rtol=1e-5)


def test_depth_of_uniform_depth_scene_is_coverage_times_depth():
    """All Gaussians at one depth z: the expected depth is z (1 - T_final) at every pixel."""
    scene = synth.uniform_scene(2000, 0, seed=6)
    scene.means[:, 2] = 3.25
    cam = _cam(64, 48)
    rec, rect, _ = oracle.preprocess(scene, cam, 16)
    img = oracle.render(rec, rect, cam, 16)
    np.testing.assert_allclose(img.depth, 3.25 * (1.0 - img.t_final), atol=2e-5)


def test_weight_sum_and_white_colour_invariant():
    """With every colour 1, C = sum_i alpha_i T_i = 1 - T_final (and C <= 1 - T_final in general)."""
    scene = synth.uniform_scene(3000, 0, seed=2)
    scene.sh[:, 0, :] = 0.5 / (0.5 / math.sqrt(math.pi))
    cam = _cam(96, 80)
    rec, rect, _ = oracle.preprocess(scene, cam, 16)
    np.testing.assert_allclose(rec[rec[:, 11] > 0, 6:9], 1.0, atol=1e-6)
    img = oracle.render(rec, rect, cam, 16)
    for ch in range(3):
        np.testing.assert_allclose(img.rgb[:, ch], 1.0 - img.t_final, atol=1e-5)
    scene2 = synth.uniform_scene(3000, 0, seed=2)
    rec2, rect2, _ = oracle.preprocess(scene2, cam, 16)
    img2 = oracle.render(rec2, rect2, cam, 16)
    assert np.all(img2.rgb.max(axis=1) <= rec2[:, 6:9].max() * (1.0 - img2.t_final) + 1e-5)
    assert np.all(img2.t_final > 0) and np.all(img2.t_final <= 1)


def test_input_order_invariance():
    scene = synth.uniform_scene(4000, 1, seed=9)
    cam = _cam(80, 64, yaw=4.0)
    rec, rect, _ = oracle.preprocess(scene, cam, 16)
    assert len(np.unique(rec[rec[:, 11] > 0, 9])) == int((rec[:, 11] > 0).sum())   # no depth ties
    img = oracle.render(rec, rect, cam, 16)
    perm = np.random.default_rng(1).permutation(scene.n)
    rec_p, rect_p, _ = oracle.preprocess(scene.subset(perm), cam, 16)
    img_p = oracle.render(rec_p, rect_p, cam, 16)
    assert np.array_equal(img.rgb, img_p.rgb)
    assert np.array_equal(img.t_final, img_p.t_final)


@pytest.mark.parametrize("seed,deg", [(21, 0), (22, 3), (23, 1)])
def test_fp64_brute_force_tiny_scene(seed, deg):
    scene = synth.uniform_scene(64, deg, seed=seed, log_scale_mean=-2.2)
    cam = synth.pinhole_camera(32, 32, 90.0, 3.0, 0.01)
    rec, rect, _ = oracle.preprocess(scene, cam, 8)
    img = oracle.render(rec, rect, cam, 8)
    ref, tref, p = brute_fp64.render64(scene, cam, 8)
    vis = rec[:, 11] > 0
    assert np.array_equal(vis, p["visible"])
    assert vis.sum() > 20
    assert np.array_equal(rect[vis], p["rect"][vis])
    np.testing.assert_allclose(rec[vis, 9], p["depth"][vis], rtol=1e-6)
    np.testing.assert_allclose(rec[vis, 6:9], p["rgb"][vis], atol=2e-6)
    ok = img.margin >= 1e-4
    assert ok.mean() > 0.9
    err = np.abs(img.rgb - ref.reshape(-1, 3)).max(axis=1)
    assert err[ok].max() < 1e-5, err[ok].max()
    assert np.abs(img.t_final - tref.reshape(-1))[ok].max() < 1e-5
    # the work counts of the composite (the flop count's n_eval and n_contrib)
    assert np.array_equal(img.n_eval[ok], p["n_eval"].reshape(-1)[ok])
    assert np.array_equal(img.n_blend[ok], p["n_blend"].reshape(-1)[ok])
    assert (img.n_blend <= img.n_eval).all() and img.n_blend.sum() > 0


# ------------------------------------------------------------------ keys, ranges
def test_keys_brute_force_membership_and_order():
    scene = synth.uniform_scene(3000, 0, seed=5)
    cam = _cam(128, 96, yaw=2.0)
    B = 16
    rec, rect, touched = oracle.preprocess(scene, cam, B)
    tx_n, ty_n = oracle.tiles(128, B), oracle.tiles(96, B)
    keys, vals = oracle.sorted_keys(rec, rect, tx_n)
    assert len(keys) == int(touched.sum())
    expect = []
    for g in range(scene.n):
        if rec[g, 11] == 0:
            continue
        u, v, r = float(rec[g, 0]), float(rec[g, 1]), float(rec[g, 10])
        db = int(np.float32(rec[g, 9]).view(np.uint32))
        for ty in range(ty_n):
            for tx in range(tx_n):
                # tile [tB, tB+B) intersects the 3-sigma square [u-r, u+r] x [v-r, v+r]
                if tx * B <= u + r and tx * B + B > u - r and ty * B <= v + r and ty * B + B > v - r:
                    expect.append(((ty * tx_n + tx) << 32 | db, g))
    expect.sort()
    assert [int(k) for k in keys] == [k for k, _ in expect]
    assert [int(v) for v in vals] == [g for _, g in expect]
    ranges = oracle.tile_ranges(keys, tx_n * ty_n)
    for t in range(tx_n * ty_n):
        idx = [j for j, (k, _) in enumerate(expect) if k >> 32 == t]
        if idx:
            assert (ranges[t, 0], ranges[t, 1]) == (idx[0], idx[-1] + 1)
        else:
            assert ranges[t, 0] == ranges[t, 1]


def test_depth_bits_order_equals_depth_order():
    scene = synth.uniform_scene(2000, 0, seed=8)
    rec, _, _ = oracle.preprocess(scene, _cam(), 16)
    d = rec[rec[:, 11] > 0, 9]
    bits = d.view(np.uint32)
    assert np.array_equal(np.argsort(d, kind="stable"), np.argsort(bits, kind="stable"))


# ------------------------------------------------------------------ foveation
def test_foveal_radius_eq1_uses_paper_theta():
    g = json.load(open(GOLDEN))
    theta = g["theta_i_deg"]["value"]
    cam = _cam(256, 256)
    fv = oracle.fovea(theta_deg=(theta, 36.0), dtheta_deg=0.0)
    r2 = oracle.layer_radii2(cam, fv)
    np.testing.assert_allclose(math.sqrt(r2[0]), 128 * math.tan(math.radians(18.0)), rtol=1e-6)
    fv2 = oracle.fovea(theta_deg=(theta, 36.0), dtheta_deg=2.1)
    np.testing.assert_allclose(math.sqrt(oracle.layer_radii2(cam, fv2)[0]),
                               128 * math.tan(math.radians(20.1)), rtol=1e-6)


@pytest.mark.parametrize("gaze", [(127.5, 127.5), (3.0, 250.0), (200.2, 60.7), (-40.0, 128.0)])
def test_level_map_brute_force_geometry(gaze):
    cam = _cam(256, 240)
    B = 16
    fv = oracle.fovea()
    lv = oracle.level_map(cam, B, fv, gaze)
    r = [128 * math.tan(math.radians(18.0)), 128 * math.tan(math.radians(36.0))]
    tx_n, ty_n = oracle.tiles(256, B), oracle.tiles(240, B)
    for ty in range(ty_n):
        for tx in range(tx_n):
            xs = np.arange(tx * B, min(tx * B + B, 256))
            ys = np.arange(ty * B, min(ty * B + B, 240))
            X, Y = np.meshgrid(xs, ys)
            d = np.sqrt((X - gaze[0]) ** 2 + (Y - gaze[1]) ** 2).min()
            expect = 4 if d <= r[0] else (2 if d <= r[1] else 1)
            if min(abs(d - r[0]), abs(d - r[1])) < 1e-3:
                continue
            assert lv[ty * tx_n + tx] == expect, (tx, ty, d)


def test_level4_tile_count_at_centre_closed_form():
    """Centre gaze on a 256^2 image: count tiles whose nearest point lies in the disc."""
    cam = _cam(256, 256)
    lv = oracle.level_map(cam, 16, oracle.fovea(), (127.5, 127.5))
    r = 128 * math.tan(math.radians(18.0))
    count = 0
    for ty in range(16):
        for tx in range(16):
            # distance from the centre (127.5, 127.5) to the tile's pixel-centre box
            dx = max(tx * 16 - 127.5, 127.5 - (tx * 16 + 15), 0.0)
            dy = max(ty * 16 - 127.5, 127.5 - (ty * 16 + 15), 0.0)
            count += dx * dx + dy * dy <= r * r
    assert int((lv == 4).sum()) == count
    assert count == 32      # 4 centre tiles + rings: fixed by r = 41.6 px and B = 16


def test_foveated_live_pixels_equal_full_and_dead_inherit_top_left():
    g = json.load(open(GOLDEN))
    assert g["peripheral_rendered_pixel"]["value"] == "top-left"
    w = synth.small_single_view()
    scene = w.scene.subset(np.arange(4000))
    cam = w.cameras(0)[0]
    rec, rect, _ = oracle.preprocess(scene, cam, 16)
    full = oracle.render(rec, rect, cam, 16)
    lv = oracle.level_map(cam, 16, oracle.fovea(), w.fixed_gaze_px)
    fov = oracle.render(rec, rect, cam, 16, level=lv)
    H = W = 256
    rgb_f = full.rgb.reshape(H, W, 3)
    rgb_v = fov.rgb.reshape(H, W, 3)
    live = fov.rendered.reshape(H, W).astype(bool)
    assert np.array_equal(rgb_v[live], rgb_f[live])
    tl = rgb_f[0::2, 0::2]
    inherited = np.repeat(np.repeat(tl, 2, axis=0), 2, axis=1)
    assert np.array_equal(rgb_v[~live], inherited[~live])
    # pixel density per level: level k renders exactly k of the 4 pixels of each block
    for t in range(256):
        ty, tx = divmod(t, 16)
        blk = live[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16]
        assert blk.sum() == 64 * int(lv[t])
        assert blk[0::2, 0::2].all()          # top-left always rendered
    # peripheral (level 1) tiles render only top-left pixels
    for t in np.nonzero(lv == 1)[0]:
        ty, tx = divmod(int(t), 16)
        blk = live[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16]
        assert not blk[1::2, :].any() and not blk[:, 1::2].any()
    # level 2 is the checkerboard TL + BR
    for t in np.nonzero(lv == 2)[0]:
        ty, tx = divmod(int(t), 16)
        blk = live[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16]
        assert blk[1::2, 1::2].all() and not blk[0::2, 1::2].any() and not blk[1::2, 0::2].any()


def test_pixel_list_mode_matches_full_image():
    w = synth.small_single_view()
    scene = w.scene.subset(np.arange(3000))
    cam = w.cameras(0)[0]
    rec, rect, _ = oracle.preprocess(scene, cam, 16)
    lv = oracle.level_map(cam, 16, oracle.fovea(), w.fixed_gaze_px)
    full = oracle.render(rec, rect, cam, 16, level=lv)
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(0, 256, 500), rng.integers(0, 256, 500)], axis=1)
    part = oracle.render(rec, rect, cam, 16, level=lv, pixels=pix)
    flat = pix[:, 1] * 256 + pix[:, 0]
    assert np.array_equal(part.rgb, full.rgb[flat])
    assert np.array_equal(part.rendered, full.rendered[flat])


def test_interpolating_fill_reproduces_a_linear_ramp():
    """A linear image sampled on the rendered pixels is reproduced exactly (up to fp32
    rounding) at interior skipped pixels: the mean of two or four symmetric neighbours of a
    linear function is its value at the centre."""
    H, W = 12, 16
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float32)
    ramp = np.stack([0.01 * xs + 0.02 * ys, 0.5 - 0.01 * xs, 0.03 * ys], -1).astype(np.float32)
    lab = np.where((xs % 2) == (ys % 2), np.where(xs % 2 == 0, 1, 2), np.where(xs % 2 == 1, 3, 4))
    for level in (1, 2, 3):
        rendered = lab <= level
        img = ramp.copy()
        img[~rendered] = 0.0                      # whatever the skipped pixels held
        out = oracle.fill_interpolate(img, rendered)
        assert np.array_equal(out[rendered], ramp[rendered])
        interior = ~rendered
        interior[0, :] = interior[-1, :] = False
        interior[:, 0] = interior[:, -1] = False
        np.testing.assert_allclose(out[interior], ramp[interior], atol=2e-6)


def test_interpolating_fill_edge_rules():
    """Neighbours outside the image or skipped do not count; a pixel without rendered
    4-neighbours uses its rendered diagonals; with none, it keeps its value."""
    img = np.zeros((3, 3, 3), np.float32)
    rendered = np.zeros((3, 3), bool)
    img[0, 0] = 1.0
    img[2, 2] = 3.0
    rendered[0, 0] = rendered[2, 2] = True
    out = oracle.fill_interpolate(img, rendered)
    np.testing.assert_array_equal(out[1, 1], np.float32(2.0))     # diagonals (0,0) and (2,2)
    np.testing.assert_array_equal(out[0, 1], np.float32(1.0))     # left neighbour only
    img2 = np.full((1, 1, 3), 7.0, np.float32)
    np.testing.assert_array_equal(oracle.fill_interpolate(img2, np.zeros((1, 1), bool)), img2)


def _ranges_of(counts):
    ends = np.cumsum(counts).astype(np.uint32)
    return np.stack([ends - np.asarray(counts, np.uint32), ends], axis=1)


def test_count_levels_hand_counted():
    """Count-based tile levels (Sec. 3.6 / 4.6 reading): the k = floor(frac * tiles) heaviest
    tiles at level 2 or 3 drop one level; hand-counted expectations."""
    counts = [5, 0, 9, 9, 3, 7, 1, 0]
    level = np.array([2, 2, 3, 2, 4, 1, 3, 2], np.uint8)
    r = _ranges_of(counts)
    cases = {
        0.0: [2, 2, 3, 2, 4, 1, 3, 2],     # off
        0.1: [2, 2, 3, 2, 4, 1, 3, 2],     # k = 0
        0.25: [2, 2, 2, 1, 4, 1, 3, 2],    # k = 2: tau = 9, both 9s drop
        0.375: [2, 2, 2, 1, 4, 1, 3, 2],   # k = 3: tau = 7 hits a level-1 tile (kept)
        0.5: [1, 2, 2, 1, 4, 1, 3, 2],     # k = 4: tau = 5
        1.0: [1, 2, 2, 1, 4, 1, 2, 2],     # k = tiles: every non-empty tile, empty ones kept
    }
    for frac, want in cases.items():
        got = oracle.count_levels(level, r, frac)
        assert got.tolist() == want, (frac, got)
    assert level.tolist() == [2, 2, 3, 2, 4, 1, 3, 2]      # input untouched


def test_count_levels_ties_and_fp32_k():
    """Ties at tau are all heavy (more than k tiles may drop); k is taken in fp32 like the
    kernel: 0.7f * 10 rounds to 7.0f, where the same fp32 fraction multiplied in fp64 gives
    6.9999999 and k = 6."""
    r = _ranges_of([4, 4, 4, 1])
    assert oracle.count_levels(np.full(4, 3, np.uint8), r, 0.25).tolist() == [2, 2, 2, 3]
    counts = list(range(10, 0, -1))                      # 10, 9, ..., 1
    got = oracle.count_levels(np.full(10, 2, np.uint8), _ranges_of(counts), 0.7)
    assert got.tolist() == [1] * 7 + [2] * 3
    assert int(np.floor(float(np.float32(0.7)) * 10)) == 6   # the fp64 product would keep 6
