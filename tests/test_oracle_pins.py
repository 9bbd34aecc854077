"""Pins of the FP64 oracle against closed forms, library routines, invariants and brute force.

Each test fixes a result by something other than the oracle's own formulas:
* Sec. 3 (first equation, projection): closed forms of the 2D covariance for isotropic and
  axis-aligned Gaussians, and Sigma' against a finite-difference Jacobian of the pinhole map
  with the rotation from scipy (scalar-last quaternion convention).
* Sec. 3 (second equation, compositing): two-layer "over" and k identical layers.
* Sec. 3 (Blinn-Phong): n parallel / perpendicular to l, beta -> 0, a 45-degree half vector.
* Sec. 4.5 (composition and edits): spatially disjoint models, hidden models, zero opacity
  scale, affinity in the palette colour.
* Brute force over all Gaussians per pixel on tiny scenes (no tiles, lists or key sort).
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import scenegen as sg
from oracle import brute
from tests._util import axis_camera, cat_models, single_model


def _proj1(model, cam, lowpass=oracle.LOWPASS, edits=None):
    edits = sg.identity_edits([model]) if edits is None else edits
    comp = oracle.compose([model])
    return oracle.project(comp, oracle.edit_table(edits), cam, lowpass)


@pytest.mark.parametrize("lowpass", [0.0, 0.3])
@pytest.mark.parametrize("sigma", [0.004, 0.011, 0.05])
def test_isotropic_on_axis(lowpass, sigma):
    cam = axis_camera(W=64, H=64, z=3.0)
    m = single_model([0, 0, 0], log_scale=[math.log(sigma)] * 3, quat=[0.3, -0.2, 0.5, 0.7])
    p = _proj1(m, cam, lowpass)
    sigma = math.exp(float(m.log_scale[0, 0]))  # the stored (float32) log-scale
    s2 = (cam.fx * sigma / 3.0) ** 2 + lowpass
    assert p.cov[0] == pytest.approx([s2, 0.0, s2], rel=1e-12, abs=1e-12)
    assert p.conic[0] == pytest.approx([1 / s2, 0.0, 1 / s2], rel=1e-12, abs=1e-12)
    assert p.radius[0] == math.ceil(3.0 * math.sqrt(s2))
    assert p.uv[0] == pytest.approx([32.0, 32.0], abs=1e-12)
    assert p.depth[0] == pytest.approx(3.0)


def _rn32(q):
    """The float32 nearest to the rational q (ties to even), decided in exact arithmetic."""
    from fractions import Fraction
    f = np.float32(float(q))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    return min(cands, key=lambda c: (abs(Fraction(float(c)) - q), int(np.float32(c).view(np.uint32)) & 1))


def test_depth_key_is_the_exact_camera_z_rounded_once():
    """The depth that keys the sort is the camera-space z of the (float32) mean, R_z . mu + t_z,
    in float64 (within 4 ulp of float64 of the exact rational value), and its float32 key is the
    exact value rounded once to the nearest float32 wherever the oracle does not certify it as
    near a rounding midpoint (depth_margin); the near-plane decision follows the exact z; and
    along every tile list of a scene with many close depths the exact rational depths never
    decrease (the order the sort produces is the order of the true depths)."""
    from fractions import Fraction
    rng = np.random.default_rng(12)
    w = sg.tiny_scene(300, 32, 32, 3, n_models=1)
    comp = oracle.compose(w.models)
    table = oracle.edit_table(w.edits)
    checked, culled, certified = 0, 0, 0
    for dist in (3.0, 3.0, 0.6, 0.6):  # the close cameras put part of the scene behind the near plane
        cam = sg.look_at(dist * sg.random_direction(rng), 32, 32)
        p = oracle.project(comp, table, cam)
        R = np.asarray(cam.R, np.float32).reshape(3, 3)
        t2 = Fraction(float(np.float32(cam.t[2])))
        exact_z = []
        for g in range(comp.n):
            mu = comp.mean[g].astype(np.float32)
            terms = [Fraction(float(R[2, j])) * Fraction(float(mu[j])) for j in range(3)] + [t2]
            exact = sum(terms)
            exact_z.append(exact)
            mag = float(sum(abs(x) for x in terms))
            assert abs(float(Fraction(float(p.depth[g])) - exact)) <= 4 * 2.0 ** -53 * mag, g
            if p.radius[g] > 0:
                if p.depth_margin[g] < 2.0 ** -40:
                    certified += 1
                else:
                    assert np.float32(p.depth[g]) == _rn32(exact), g
                checked += 1
            if exact <= Fraction(cam.znear):
                assert p.radius[g] == 0, g  # behind the near plane
                culled += 1
        # order along the tile lists of this view (float32 keys from the float64 depth)
        b = oracle.bin_pairs(*oracle.decision_inputs([p]), [(cam.W, cam.H)])
        for a, e in b.ranges:
            zs = [exact_z[int(v)] for v in b.values[a:e]]
            assert all(z0 <= z1 for z0, z1 in zip(zs, zs[1:]))
    assert checked > 500 and culled > 20 and certified == 0, (checked, culled, certified)


def test_depth_margin_flags_values_near_a_rounding_midpoint():
    """A Gaussian whose camera z is a float32 midpoint gets a depth margin of 0; one whose z is a
    float32 value gets the largest, half an ulp (relative to |t_z| + sum |R_zk mu_k| = z)."""
    z32 = np.float32(3.0)
    mid = (float(z32) + float(np.nextafter(z32, np.float32(np.inf)))) / 2.0
    m = single_model([0.0, 0.0, 0.0], log_scale=[-3.0] * 3)
    for z, want in ((mid, 0.0), (float(z32), 0.5 * float(np.spacing(z32)) / float(z32))):
        c = axis_camera(W=32, H=32, z=3.0)
        c.t = np.array([0.0, 0.0, z])  # float64: the oracle takes the camera as given
        p = _proj1(m, c, 0.3)
        assert p.radius[0] > 0 and p.depth[0] == z
        assert p.depth_margin[0] == pytest.approx(want, rel=1e-9, abs=1e-18)



def test_axis_aligned_and_quarter_turn():
    cam = axis_camera(W=64, H=64, z=4.0)
    ls = np.log(np.array([0.02, 0.005, 0.03])).astype(np.float32)
    sx, sy, sz = np.exp(ls.astype(np.float64))
    p = _proj1(single_model([0, 0, 0], log_scale=ls), cam, 0.3)
    fz = cam.fx / 4.0
    assert p.cov[0] == pytest.approx([(fz * sx) ** 2 + 0.3, 0.0, (fz * sy) ** 2 + 0.3], rel=1e-12, abs=1e-14)
    c45 = math.cos(math.pi / 4)
    p2 = _proj1(single_model([0, 0, 0], log_scale=ls, quat=[c45, 0, 0, c45]), cam, 0.3)
    assert p2.cov[0] == pytest.approx([(fz * sy) ** 2 + 0.3, 0.0, (fz * sx) ** 2 + 0.3], rel=1e-6, abs=1e-9)


def test_covariance_matches_fd_jacobian_and_scipy_rotation():
    rng = np.random.default_rng(11)
    cams = [sg.look_at(3.0 * sg.random_direction(rng), 256, 192) for _ in range(4)]
    for cam in cams:
        for _ in range(8):
            mu = rng.uniform(-0.5, 0.5, 3)
            q = rng.standard_normal(4)
            ls = rng.normal(-4.0, 0.5, 3)
            m = single_model(mu, log_scale=ls, quat=q)
            p = _proj1(m, cam, 0.0)
            qf = np.asarray(m.quat[0], np.float64)
            Rq = Rotation.from_quat([qf[1], qf[2], qf[3], qf[0]]).as_matrix()
            Sig = Rq @ np.diag(np.exp(2.0 * np.asarray(m.log_scale[0], np.float64))) @ Rq.T
            Rw = np.asarray(cam.R, np.float64).reshape(3, 3)
            mc = Rw @ np.asarray(m.mean[0], np.float64) + np.asarray(cam.t, np.float64)

            def pin(xc):
                return np.array([cam.fx * xc[0] / xc[2] + cam.cx, cam.fy * xc[1] / xc[2] + cam.cy])

            h = 1e-6
            J = np.stack([(pin(mc + h * e) - pin(mc - h * e)) / (2 * h) for e in np.eye(3)], 1)
            cov = J @ Rw @ Sig @ Rw.T @ J.T
            assert p.cov[0] == pytest.approx([cov[0, 0], cov[0, 1], cov[1, 1]], rel=2e-6, abs=1e-9)
            assert p.uv[0] == pytest.approx(pin(mc), rel=1e-12)


def test_culling_near_plane_and_hidden_model():
    cam = axis_camera(z=0.1)  # the point is 0.1 in front of the camera: behind the 0.2 near plane
    assert _proj1(single_model([0, 0, 0]), cam).radius[0] == 0
    cam = axis_camera(z=3.0)
    m = single_model([0, 0, 0])
    ed = sg.identity_edits([m])
    ed.visible[0] = 0
    assert _proj1(m, cam, edits=ed).radius[0] == 0


# ------------------------------------------------------------------ shading (Blinn-Phong)
def _rgb(m, cam, edits=None):
    return _proj1(m, cam, edits=edits).rgb[0]


def test_shading_headlight_normal_parallel():
    cam = axis_camera(z=3.0)
    alb = np.array([0.2, 0.5, 0.9])
    m = single_model([0, 0, 0], albedo=alb, normal=[0, 0, -1])  # normal points at the camera
    ka, kd, ks, _ = sg.KADS_DEFAULT
    assert _rgb(m, cam) == pytest.approx((ka + kd) * alb + ks, rel=1e-6)
    m2 = single_model([0, 0, 0], albedo=alb, normal=[0, 0, 5])  # unnormalised, facing away: |n.l|
    assert _rgb(m2, cam) == pytest.approx((ka + kd) * alb + ks, rel=1e-6)


def test_shading_normal_perpendicular_is_ambient_only():
    cam = axis_camera(z=3.0)
    alb = np.array([0.3, 0.6, 0.1])
    m = single_model([0, 0, 0], albedo=alb, normal=[1, 0, 0])
    cv = m.palette.astype(np.float64) + m.dcolor[0].astype(np.float64)  # stored c_p + dc
    assert _rgb(m, cam) == pytest.approx(float(np.float32(0.2)) * cv, rel=1e-12, abs=1e-15)


def test_shading_orbital_half_vector_and_beta():
    cam = axis_camera(z=3.0, headlight=False, light_dir=[1, 0, 0])
    alb = np.array([0.4, 0.4, 0.4])
    # v = (0,0,-1) towards the camera, l = (1,0,0), n = l: n.l = 1, n.h = 1/sqrt(2)
    m = single_model([0, 0, 0], albedo=alb, normal=[1, 0, 0], kads=[0.2, 0.7, 0.3, 1.0])
    cv = m.palette.astype(np.float64) + m.dcolor[0].astype(np.float64)
    ka, kd, ks = (float(np.float32(x)) for x in (0.2, 0.7, 0.3))
    assert _rgb(m, cam) == pytest.approx((ka + kd) * cv + ks / math.sqrt(2.0), rel=1e-12)
    m0 = single_model([0, 0, 0], albedo=alb, normal=[1, 0, 0], kads=[0.2, 0.7, 0.3, 0.0])
    assert _rgb(m0, cam) == pytest.approx((ka + kd) * cv + ks, rel=1e-12)


def test_light_magnitude_edit():
    cam = axis_camera(z=3.0)
    alb = np.array([0.2, 0.5, 0.9])
    m = single_model([0, 0, 0], albedo=alb, normal=[0, 0, -1])
    ed = sg.identity_edits([m])
    ed.lam = np.array([2.0, 0.5, 3.0, 1.0], np.float32)
    ed.bias = np.array([0.1, 0.0, -0.2, 0.0], np.float32)
    ka, kd, ks = 2 * 0.2 + 0.1, 0.5 * 0.7, 3 * 0.3 - 0.2
    assert _rgb(m, cam, ed) == pytest.approx((ka + kd) * alb + ks, rel=1e-6)


def test_palette_edit_replaces_cp():
    cam = axis_camera(z=3.0)
    alb = np.array([0.2, 0.5, 0.9])
    m = single_model([0, 0, 0], albedo=alb, palette=[0.4, 0.4, 0.4], normal=[1, 0, 0])
    ed = sg.identity_edits([m])
    ed.palette[0] = [0.9, 0.1, 0.0]
    cp = np.asarray(ed.palette[0], np.float64)
    cv = cp + m.dcolor[0].astype(np.float64)
    assert _rgb(m, cam, ed) == pytest.approx(float(np.float32(0.2)) * cv, rel=1e-12, abs=1e-15)


# ------------------------------------------------------------------ compositing closed forms
def _records(uv, conic, opacity, rgb):
    return oracle.Projected(uv=np.asarray(uv, float).reshape(-1, 2), cov=np.zeros((len(opacity), 3)),
                            conic=np.asarray(conic, float).reshape(-1, 3), opacity=np.asarray(opacity, float),
                            rgb=np.asarray(rgb, float).reshape(-1, 3), depth=np.arange(1, len(opacity) + 1.0),
                            radius=np.full(len(opacity), 3, np.int32), radius_margin=np.ones(len(opacity)))


def _blend(p, px, bg=(0, 0, 0)):
    cam = sg.Camera(W=32, H=32, fx=1, fy=1, cx=16, cy=16, R=np.eye(3).reshape(9), t=np.zeros(3),
                    campos=np.zeros(3))
    return oracle.render_pixels(p, cam, np.array([px]), bg=bg)


def test_peak_alpha_and_clamp():
    for o, expect in [(0.5, 0.5), (0.98, 0.98), (0.995, 0.99), (3.0, 0.99)]:
        p = _records([[10.5, 7.5]], [[0.2, 0.0, 0.2]], [o], [[1.0, 0.5, 0.25]])
        rgba, T, last, _ = _blend(p, (10, 7))
        assert rgba[0, 3] == pytest.approx(expect, abs=1e-15)
        assert rgba[0, :3] == pytest.approx(np.array([1.0, 0.5, 0.25]) * expect, abs=1e-15)
        assert last[0] == 1


@pytest.mark.parametrize("side", [+1, -1])
def test_alpha_cutoff_1_over_255(side):
    a = 0.25
    o = 0.8
    target = (1.0 / 255.0) * (1.0 + side * 1e-6)
    d = math.sqrt(2.0 * math.log(o / target) / a)  # alpha = o exp(-a d^2 / 2) == target
    p = _records([[10.5 + d, 7.5]], [[a, 0.0, a]], [o], [[1.0, 1.0, 1.0]])
    rgba, T, last, _ = _blend(p, (10, 7))
    if side > 0:
        assert last[0] == 1 and rgba[0, 3] == pytest.approx(target, rel=1e-9)
    else:
        assert last[0] == 0 and rgba[0, 3] == 0.0


def test_two_layer_over():
    c1, c2, bg = np.array([1.0, 0.2, 0.1]), np.array([0.1, 0.9, 0.3]), np.array([0.05, 0.1, 0.7])
    p = _records([[10.5, 7.5], [10.5, 7.5]], [[0.2, 0, 0.2]] * 2, [0.6, 0.3], [c1, c2])
    rgba, T, last, _ = _blend(p, (10, 7), bg=bg)
    a1, a2 = 0.6, 0.3
    assert rgba[0, :3] == pytest.approx(a1 * c1 + (1 - a1) * a2 * c2 + (1 - a1) * (1 - a2) * bg, abs=1e-15)
    assert T[0] == pytest.approx((1 - a1) * (1 - a2), abs=1e-15)
    assert rgba[0, 3] == pytest.approx(1 - T[0], abs=1e-15)


@pytest.mark.parametrize("alpha", [0.1, 0.37, 0.5, 0.9, 0.99])
def test_k_identical_layers_termination(alpha):
    k = 200
    p = _records([[10.5, 7.5]] * k, [[0.2, 0, 0.2]] * k, [alpha] * k, [[1.0, 1.0, 1.0]] * k)
    rgba, T, last, _ = _blend(p, (10, 7))
    kk = max(j for j in range(k + 1) if (1 - alpha) ** j >= 1e-4)  # largest count keeping T >= 1e-4
    assert last[0] == kk
    assert T[0] == pytest.approx((1 - alpha) ** kk, rel=1e-12)
    assert rgba[0, 0] == pytest.approx(1 - (1 - alpha) ** kk, rel=1e-12)


def test_transmittance_monotone_over_prefixes():
    rng = np.random.default_rng(5)
    n = 40
    p = _records(np.c_[10.5 + rng.normal(0, 2, n), 7.5 + rng.normal(0, 2, n)],
                 np.c_[rng.uniform(0.05, 0.3, n), rng.uniform(-0.02, 0.02, n), rng.uniform(0.05, 0.3, n)],
                 rng.uniform(0.05, 0.9, n), rng.random((n, 3)))
    cam = sg.Camera(W=32, H=32, fx=1, fy=1, cx=16, cy=16, R=np.eye(3).reshape(9), t=np.zeros(3), campos=np.zeros(3))
    Ts = []
    for k in range(1, n + 1):
        sub = oracle.Projected(p.uv[:k], p.cov[:k], p.conic[:k], p.opacity[:k], p.rgb[:k], p.depth[:k],
                               p.radius[:k], p.radius_margin[:k])
        Ts.append(oracle.render_pixels(sub, cam, np.array([(10, 7)]))[1][0])
    assert all(b <= a for a, b in zip(Ts, Ts[1:]))
    assert Ts[-1] >= 1e-4


# ------------------------------------------------------------------ tiled oracle vs brute force
@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("headlight", [True, False])
def test_tiled_matches_brute_force(seed, headlight):
    w = sg.tiny_scene(48, 40, 24, seed, log_scale_mu=-2.6, headlight=headlight, n_models=2)
    bg = np.array([0.1, 0.2, 0.3])
    r = oracle.render(w.models, w.edits, w.cameras, bg=bg)
    p = r.projs[0]
    ref = brute.render_view(p.uv, p.conic, p.opacity, p.rgb, p.depth, p.radius, 40, 24, bg=bg)
    assert (p.radius > 0).sum() > 20
    assert r.images[0][..., 3].max() > 0.5
    np.testing.assert_allclose(r.images[0], ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.images[0][..., 3], 1.0 - r.final_T[0], rtol=0, atol=0)


def test_sampled_pixels_match_full_render():
    w = sg.tiny_scene(300, 96, 64, 3, log_scale_mu=-3.0, n_models=3)
    r = oracle.render(w.models, w.edits, w.cameras)
    rng = np.random.default_rng(0)
    pix = np.c_[rng.integers(0, 96, 200), rng.integers(0, 64, 200)]
    rgba, T, last, _ = oracle.render_pixels(r.projs[0], w.cameras[0], pix)
    np.testing.assert_array_equal(rgba, r.images[0][pix[:, 1], pix[:, 0]])
    np.testing.assert_array_equal(last, r.last[0][pix[:, 1], pix[:, 0]])


def test_sampled_pixels_backward_matches_full_backward():
    """The sampled-pixel reverse mode (used for the full-size gradient checks) equals the
    whole-image reverse mode for a dL/dRGBA that is zero outside the sampled pixels: attribute,
    edit and light gradients, on a composed scene with edits and an orbital view."""
    base = sg.tiny_scene(300, 64, 48, 9, log_scale_mu=-2.8, n_models=2)
    r0 = np.random.default_rng(11)
    cams = [base.cameras[0], sg.look_at(3.0 * sg.random_direction(r0), 48, 40, headlight=False,
                                        light_dir=sg.random_direction(r0).astype(np.float32))]
    ed = sg.random_edits(base.models, seed=12)
    ed.lam = np.array([1.2, 0.8, 1.1, 0.9], np.float32)
    ed.bias = np.array([0.03, -0.02, 0.05, 0.7], np.float32)
    bg = np.array([0.1, 0.2, 0.3])
    r = oracle.render(base.models, ed, cams, bg=bg)
    rng = np.random.default_rng(13)
    pix, dls_s, dls_full = [], [], []
    for c in cams:
        flat = rng.choice(c.W * c.H, 150, replace=False)  # distinct pixels
        p = np.c_[flat % c.W, flat // c.W]
        d = rng.normal(0, 1, (len(flat), 4))
        full = np.zeros((c.H, c.W, 4))
        full[p[:, 1], p[:, 0]] = d
        pix.append(p); dls_s.append(d); dls_full.append(full)
    g_full = oracle.render_backward(r, cams, dls_full, bg=bg)
    g_s = oracle.pixels_backward(r.comp, r.table, cams, r.projs, pix, dls_s, bg=bg)
    for k in oracle.PARAMS:
        a, b = g_s.params[k], g_full.params[k]
        assert np.abs(b).max() > 0, k
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-10 * np.abs(b).max(), err_msg=k)
    np.testing.assert_allclose(g_s.edit, g_full.edit, rtol=0, atol=1e-10 * np.abs(g_full.edit).max())
    np.testing.assert_allclose(g_s.light, g_full.light, rtol=0, atol=1e-10 * np.abs(g_full.light).max())
    assert np.abs(g_full.light[1]).max() > 0


@pytest.mark.parametrize("headlight", [True, False])
def test_rigid_motion_of_scene_and_camera_leaves_the_image_unchanged(headlight):
    """Moving the whole scene and the camera by one rigid motion x -> Q x + d (means, normals
    and an orbital light direction rotated, each quaternion composed as r q with r the
    rotation's quaternion, camera R' = R Q^T, t' = t - R Q^T d) leaves the image unchanged up to
    the float32 rounding of the moved inputs. Sec. 3's projection and shading depend only on
    relative geometry; a transposed rotation from a quaternion, a wrong composition order or a
    world-space quantity used where a camera-space one is meant breaks this."""
    import copy

    from scipy.spatial.transform import Rotation
    w = sg.tiny_scene(400, 48, 40, 21, log_scale_mu=-2.8, headlight=headlight, n_models=2)
    rot = Rotation.from_rotvec([0.3, -0.7, 0.4])
    Q = rot.as_matrix()
    x, y, z, qw = rot.as_quat()  # scalar last
    d = np.array([0.21, -0.13, 0.08])

    def compose_r(q):  # Hamilton product r q, quaternions (w, x, y, z)
        w2, x2, y2, z2 = q.T
        return np.stack([qw * w2 - x * x2 - y * y2 - z * z2, qw * x2 + x * w2 + y * z2 - z * y2,
                         qw * y2 - x * z2 + y * w2 + z * x2, qw * z2 + x * y2 - y * x2 + z * w2], 1)

    moved = []
    for m in w.models:
        c = m.copy()
        c.mean = (m.mean.astype(np.float64) @ Q.T + d).astype(np.float32)
        c.quat = compose_r(m.quat.astype(np.float64)).astype(np.float32)
        c.normal = (m.normal.astype(np.float64) @ Q.T).astype(np.float32)
        moved.append(c)
    cam = w.cameras[0]
    cam2 = copy.deepcopy(cam)
    R2 = cam.R.reshape(3, 3).astype(np.float64) @ Q.T
    cam2.R = R2.astype(np.float32).reshape(9)
    cam2.t = (cam.t.astype(np.float64) - R2 @ d).astype(np.float32)
    cam2.campos = (Q @ cam.campos.astype(np.float64) + d).astype(np.float32)
    cam2.light_dir = (Q @ cam.light_dir.astype(np.float64)).astype(np.float32)
    a = oracle.render(w.models, w.edits, [cam]).images[0]
    b = oracle.render(moved, w.edits, [cam2]).images[0]
    assert a[..., 3].max() > 0.5
    assert np.abs(a - b).max() < 1e-5


@pytest.mark.parametrize("headlight", [True, False])
def test_uniform_scaling_of_scene_and_camera_leaves_the_image_unchanged(headlight):
    """Scaling positions by 2 and the Gaussians' sizes by 2 (log-scale + ln 2), with the camera
    at twice its distance (t' = 2 t), leaves every pixel unchanged: the pinhole Jacobian J
    scales as 1/z and Sigma as s^2, so J W Sigma W^T J^T, the dilation, the radii, the depth
    order and the shading are unchanged. A Jacobian with a wrong power of z breaks this."""
    import copy
    w = sg.tiny_scene(400, 48, 40, 23, log_scale_mu=-2.8, headlight=headlight, n_models=2)
    scaled = []
    for m in w.models:
        c = m.copy()
        c.mean = (2.0 * m.mean).astype(np.float32)  # exact
        c.log_scale = (m.log_scale.astype(np.float64) + np.log(2.0)).astype(np.float32)
        scaled.append(c)
    cam = w.cameras[0]
    cam2 = copy.deepcopy(cam)
    cam2.t = (2.0 * cam.t).astype(np.float32)
    cam2.campos = (2.0 * cam.campos).astype(np.float32)
    a = oracle.render(w.models, w.edits, [cam]).images[0]
    b = oracle.render(scaled, w.edits, [cam2]).images[0]
    assert a[..., 3].max() > 0.5
    assert np.abs(a - b).max() < 1e-5


# ------------------------------------------------------------------ invariants (Sec. 4.5)
def test_spatially_disjoint_models_compose_to_union():
    a = sg.tiny_scene(30, 64, 32, 7, log_scale_mu=-3.2).models[0]
    b = sg.tiny_scene(30, 64, 32, 8, log_scale_mu=-3.2).models[0]
    cam = axis_camera(W=64, H=32, z=3.0)
    # push a to the left third and b to the right third of the image (tiles never shared)
    a.mean[:, 0] = a.mean[:, 0] * 0.25 - 0.75
    b.mean[:, 0] = b.mean[:, 0] * 0.25 + 0.75
    a.mean[:, 1] *= 0.3
    b.mean[:, 1] *= 0.3
    ra = oracle.render([a], sg.identity_edits([a]), [cam])
    rb = oracle.render([b], sg.identity_edits([b]), [cam])
    rab = oracle.render([a, b], sg.identity_edits([a, b]), [cam])
    ta = ra.images[0][..., 3] > 0
    tb = rb.images[0][..., 3] > 0
    assert ta.any() and tb.any() and not (ta & tb).any()
    expect = np.where(ta[..., None], ra.images[0], rb.images[0])
    np.testing.assert_array_equal(rab.images[0], expect)


def test_composition_equals_concatenated_single_model():
    w = sg.tiny_scene(60, 48, 48, 9, log_scale_mu=-3.0, n_models=3)
    ms = w.models
    flat = cat_models(ms)
    cp = np.concatenate([np.repeat(m.palette[None].astype(np.float64), m.n, 0) for m in ms])
    flat.dcolor = (cp + np.concatenate([m.dcolor for m in ms]).astype(np.float64))
    flat.palette = np.zeros(3, np.float32)
    comp = oracle.compose([flat])
    comp.dcolor = np.ascontiguousarray(flat.dcolor, np.float64)
    r1 = oracle.render(ms, w.edits, w.cameras)
    r2 = oracle.render([flat], sg.identity_edits([flat]), w.cameras, comp=comp,
                       table=oracle.edit_table(sg.Edits(np.zeros((1, 3), np.float32), np.ones(1, np.float32),
                                                        np.ones(1, np.int32))))
    np.testing.assert_array_equal(r1.images[0], r2.images[0])


def test_hidden_model_edits_change_nothing_and_zero_opacity_scale_hides():
    w = sg.tiny_scene(60, 48, 48, 10, log_scale_mu=-3.0, n_models=3)
    ed = w.edits.copy()
    ed.visible[1] = 0
    r1 = oracle.render(w.models, ed, w.cameras)
    ed2 = ed.copy()
    ed2.palette[1] = [0.9, 0.0, 0.4]
    ed2.opacity_scale[1] = 7.0
    r2 = oracle.render(w.models, ed2, w.cameras)
    np.testing.assert_array_equal(r1.images[0], r2.images[0])
    ed3 = w.edits.copy()
    ed3.opacity_scale[1] = 0.0
    r3 = oracle.render(w.models, ed3, w.cameras)
    np.testing.assert_array_equal(r1.images[0], r3.images[0])
    assert len(r3.bins.keys) > len(r1.bins.keys)  # the lists differ, the image does not


def test_image_affine_in_palette():
    w = sg.tiny_scene(60, 48, 48, 12, log_scale_mu=-3.0, n_models=2)
    e1, e2, e3 = w.edits.copy(), w.edits.copy(), w.edits.copy()
    e1.palette[0] = [0.125, 0.25, 0.375]  # dyadic values: the midpoint is exact in float32
    e2.palette[0] = [0.875, 0.5, 0.0]
    e3.palette[0] = [0.5, 0.375, 0.1875]
    i1, i2, i3 = (oracle.render(w.models, e, w.cameras).images[0] for e in (e1, e2, e3))
    np.testing.assert_allclose(i3, 0.5 * (i1 + i2), rtol=0, atol=1e-13)


def test_camera_roll_rotates_image():
    w = sg.tiny_scene(80, 64, 64, 13, log_scale_mu=-3.0)
    cam = w.cameras[0]
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    roll = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], np.float64)  # 90 deg about the optical axis
    cam2 = sg.Camera(**{**cam.__dict__, "R": (roll @ R).astype(np.float32).reshape(9),
                        "t": (roll @ np.asarray(cam.t, np.float64)).astype(np.float32)})
    r1 = oracle.render(w.models, w.edits, [cam])
    r2 = oracle.render(w.models, w.edits, [cam2])
    # camera-space (x, y) -> (-y, x): pixel (i, j) of view 1 lands at (W-1-j, i) of view 2
    rot = np.rot90(r1.images[0], k=-1, axes=(0, 1))
    ok = np.abs(r2.images[0] - rot).max(-1) < 1e-9
    assert ok.mean() > 0.995


def test_permutation_invariance_with_distinct_depths():
    w = sg.tiny_scene(70, 48, 48, 14, log_scale_mu=-3.0)
    m = w.models[0]
    perm = np.random.default_rng(3).permutation(m.n)
    mp = sg.Model(**{k: getattr(m, k)[perm] for k in sg.ATTRS}, palette=m.palette)
    r1 = oracle.render([m], w.edits, w.cameras)
    r2 = oracle.render([mp], w.edits, w.cameras)
    assert len(np.unique(r1.projs[0].depth.astype(np.float32))) == m.n
    np.testing.assert_array_equal(r1.images[0], r2.images[0])


# ------------------------------------------------------------------ binning / ordering
@pytest.mark.parametrize("th", [16, 8])
def test_bin_matches_python_sort_with_ties(th):
    """The oracle's tile lists against a plain Python rebuild (exact rectangles, a sort by
    (tile, depth bits) with ties in emission order), for 16 x 16 and 16 x 8 tiles."""
    sizes = [(64, 48), (40, 40), (100, 30)]
    xy, rad, depth = sg.synthetic_projected(sizes, 300, seed=4)
    b = oracle.bin_pairs(xy, rad, depth, sizes, tile=(16, th))
    exp = []
    toff = 0
    for v, (W, H) in enumerate(sizes):
        gx, gy = -(-W // 16), -(-H // th)
        for g in range(300):
            r = int(rad[v, g])
            if r <= 0:
                continue
            u, vv = float(xy[v, g, 0]), float(xy[v, g, 1])
            # exact real-number rectangle (float32 inputs; r integer; u -+ r exact in float64)
            x0 = min(max(math.floor((u - r) / 16), 0), gx)
            x1 = min(max(math.floor((u + r) / 16) + 1, 0), gx)
            y0 = min(max(math.floor((vv - r) / th), 0), gy)
            y1 = min(max(math.floor((vv + r) / th) + 1, 0), gy)
            bits = int(np.float32(depth[v, g]).view(np.uint32))
            for ty in range(y0, y1):
                for tx in range(x0, x1):
                    exp.append((((toff + ty * gx + tx) << 32) | bits, len(exp), g))
        toff += gx * gy
    exp.sort(key=lambda e: (e[0], e[1]))
    assert len(exp) == len(b.keys) > 1000
    np.testing.assert_array_equal(b.keys, np.array([e[0] for e in exp], np.uint64))
    np.testing.assert_array_equal(b.values, np.array([e[2] for e in exp], np.uint32))
    tiles = b.keys >> np.uint64(32)
    for t in range(len(b.ranges)):
        s, e = b.ranges[t]
        idx = np.nonzero(tiles == t)[0]
        if len(idx):
            assert (s, e) == (idx[0], idx[-1] + 1)
        else:
            assert s == e == 0


# ------------------------------------------------------------------ auxiliary maps (Sec. 4.2, 4.3)
def test_aux_maps_reduce_to_alpha_and_colour():
    """The auxiliary compositing applies the RGB blend weights T_i alpha_i: per-Gaussian values
    (1, r, g, b) give (1 - T, C) of the colour render with a black background; a scene whose
    normals all point one way gives N = n (1 - T); the last channel is 1 - T."""
    import ctypes as C
    w = sg.tiny_scene(600, 40, 32, 71, log_scale_mu=-3.0, n_models=2)
    cams = w.cameras
    r = oracle.render(w.models, w.edits, cams, bg=(0.0, 0.0, 0.0))
    p = r.projs[0]
    c = cams[0]
    aux = np.ascontiguousarray(np.c_[np.ones(len(p.opacity)), p.rgb], np.float64)
    o = np.zeros((c.H, c.W, 5))
    oracle.lib().orc_render_view_aux(oracle._p(p.uv), oracle._p(p.conic), oracle._p(p.opacity), oracle._p(p.rgb),
                                     oracle._p(aux), C.c_int32(4), oracle._p(r.bins.values, C.c_uint32),
                                     oracle._p(r.bins.ranges, C.c_uint32), C.c_int64(0), C.c_int32(c.W),
                                     C.c_int32(c.H), C.c_int32(16), C.c_int32(16), oracle._p(o))
    img = r.images[0]
    assert img[..., 3].max() > 0.3
    np.testing.assert_allclose(o[..., 0], img[..., 3], rtol=0, atol=1e-14)
    np.testing.assert_allclose(o[..., 1:4], img[..., :3], rtol=0, atol=1e-14)
    np.testing.assert_allclose(o[..., 4], img[..., 3], rtol=0, atol=1e-15)
    # one shared normal (any length: only its direction is used)
    for m in w.models:
        m.normal[:] = np.array([0.3, -2.0, 1.1], np.float32)
    r2 = oracle.render(w.models, w.edits, cams)
    maps = oracle.render_aux(r2, cams)[0]
    n32 = np.array([0.3, -2.0, 1.1], np.float32).astype(np.float64)  # the stored (float32) normal
    n = n32 / np.linalg.norm(n32)
    np.testing.assert_allclose(maps[..., 1:4], maps[..., 11:12] * n, rtol=0, atol=1e-14)
    np.testing.assert_allclose(maps[..., 11], r2.images[0][..., 3], rtol=0, atol=1e-15)
    # depth lies between the nearest and farthest contributor's depth, times the coverage
    live = p.radius > 0
    assert np.all(maps[..., 0] <= p.depth[live].max() * maps[..., 11] + 1e-12)
    assert np.all(maps[..., 0] >= p.depth[live].min() * maps[..., 11] - 1e-12)


def test_aux_maps_of_constant_attributes():
    """With every Gaussian sharing one offset colour dc, one k = (k_a, k_d, k_s, beta) and one
    camera depth z0 (all means on the plane z_c = z0), the maps are those constants times the
    coverage 1 - T: dc (1 - T), (lambda k + b)(1 - T) with the light-magnitude edit of Sec. 4.6
    applied componentwise, and z0 (1 - T). A dropped or misplaced edit term, a wrong channel
    order or a depth other than the camera z fails one of them."""
    w = sg.tiny_scene(400, 40, 32, 72, log_scale_mu=-3.0, n_models=2)
    cam = w.cameras[0]
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    t = np.asarray(cam.t, np.float64)
    z0 = 3.0
    rng = np.random.default_rng(5)
    dc = np.array([0.12, -0.07, 0.2], np.float32)
    k = np.array([0.3, 0.6, 0.25, 12.0], np.float32)
    for m in w.models:
        xy = rng.uniform(-0.45, 0.45, (m.n, 2)) * z0 / 3.0
        xc = np.c_[xy, np.full(m.n, z0)]          # camera coordinates on the plane z_c = z0
        m.mean[:] = ((xc - t) @ R).astype(np.float32)  # world = R^T (x_c - t)
        m.dcolor[:] = dc
        m.kads[:] = k
    ed = w.edits
    ed.lam = np.array([1.3, 0.7, 1.1, 0.9], np.float32)
    ed.bias = np.array([0.05, -0.02, 0.1, 2.0], np.float32)
    r = oracle.render(w.models, ed, w.cameras)
    maps = oracle.render_aux(r, w.cameras)[0]
    cov = maps[..., 11]
    assert cov.max() > 0.3
    np.testing.assert_allclose(cov, r.images[0][..., 3], rtol=0, atol=1e-15)
    kp = ed.lam.astype(np.float64) * k.astype(np.float64) + ed.bias.astype(np.float64)
    np.testing.assert_allclose(maps[..., 4:7], cov[..., None] * dc.astype(np.float64), rtol=0, atol=1e-13)
    np.testing.assert_allclose(maps[..., 7:11], cov[..., None] * kp, rtol=0, atol=1e-12)
    # float32 storage of the means moves each camera depth by a few ulps of z0
    np.testing.assert_allclose(maps[..., 0], z0 * cov, rtol=0, atol=1e-5 * z0)
