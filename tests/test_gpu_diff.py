"""Differentiable form on the GPU against the FP64 oracle.

The oracle's held-out log-likelihood gradient (pinned on the CPU against
central finite differences and the sigma0 / Euler identities) is the
reference: dLL/dl and dLL/dsigma0 within relative 1e-4, dLL/dxyz within
1e-4 of the gradient's norm (componentwise 1e-3 relative plus 1e-5 of the
largest component), LL within relative 1e-5.  GPU central differences of LL
in l and sigma0 agree with the GPU gradient to 1e-3.
"""
import numpy as np
import pytest

from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_04631_gb300 as sbm
    sbm.load()
    return sbm


def _world(points, pose):
    """world = fp32(((r0 px + r1 py) + r2 pz) + t) in FP64 (the transform reading)."""
    T = np.asarray(pose, np.float64).reshape(4, 4)
    p = np.asarray(points, np.float32).astype(np.float64)
    out = np.empty((len(p), 3), np.float32)
    for a in range(3):
        out[:, a] = (((T[a, 0] * p[:, 0] + T[a, 1] * p[:, 1]) + T[a, 2] * p[:, 2]) + T[a, 3]).astype(np.float32)
    return out


def _params(sb, prm, **kw):
    p = sb.default_params(res=prm["res"], length_scale=prm["length_scale"], sigma0=prm["sigma0"],
                          alpha0=prm["alpha0"], free_step=prm["free_step"], num_classes=prm["num_classes"],
                          min_range=prm["min_range"], max_range=prm["max_range"], pool_blocks=1 << 14,
                          sample_capacity=1 << 21, device=0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.fixture(scope="module")
def diff_case(sb, orc):
    """Two scans of the small region (LiDAR rays thinned to 64 x 256): training sets
    from both sides (checked equal), held-out hits in world coordinates."""
    prm = dict(scenes.DIFF_PARAMS)
    scans = list(scenes.small_region_lidar_sequence(2, n_az=256))
    p = _params(sb, prm)
    op = orc.params(**prm)
    gx, gl, ox, ol, hx, hl = [], [], [], [], [], []
    with sb.Map(p) as m:
        for sc in scans:
            x, l = m.training_set(sc["points"], sc["labels"], sc["pose"])
            gx.append(x)
            gl.append(l)
    for sc in scans:
        x, l, _ = orc.training_set(op, sc["points"], sc["labels"], sc["pose"])
        ox.append(x)
        ol.append(l)
        hx.append(_world(sc["held_points"], sc["pose"]))
        hl.append(sc["held_labels"])
    gx, gl, ox, ol = map(np.concatenate, (gx, gl, ox, ol))
    order_g = np.lexsort((gl, gx[:, 2], gx[:, 1], gx[:, 0]))
    order_o = np.lexsort((ol, ox[:, 2], ox[:, 1], ox[:, 0]))
    np.testing.assert_array_equal(gx[order_g], ox[order_o])
    np.testing.assert_array_equal(gl[order_g], ol[order_o])
    return dict(prm=prm, xyz=gx, lab=gl.astype(np.int32), held=np.concatenate(hx), held_lab=np.concatenate(hl))


def _gpu_grad(sb, p, xyz, lab, held, held_lab):
    xyzl = np.concatenate([xyz, lab[:, None].astype(np.float32)], 1)
    with sb.Map(p) as m:
        m.insert_training(xyz, lab)
        m.grad_clear()
        ll = m.heldout_loglik(held, held_lab, grad=True)
        gl, gs, gx = m.backward(xyzl)
    return ll, gl, gs, gx


def test_heldout_gradient_matches_oracle(sb, orc, diff_case):
    c = diff_case
    p = _params(sb, c["prm"])
    ll, gl, gs, gx = _gpu_grad(sb, p, c["xyz"], c["lab"], c["held"], c["held_lab"])
    oll, ogl, ogs, ogx = orc.heldout_grad(orc.params(**c["prm"]), c["xyz"].astype(np.float64), c["lab"], c["held"],
                                          c["held_lab"])
    assert abs(ll - oll) <= 1e-5 * abs(oll)
    assert abs(gl - ogl) <= 1e-4 * abs(ogl), (gl, ogl)
    assert abs(gs - ogs) <= 1e-4 * abs(ogs), (gs, ogs)
    err = np.abs(gx.astype(np.float64) - ogx)
    assert np.linalg.norm(err) <= 1e-4 * np.linalg.norm(ogx)
    assert np.all(err <= 1e-3 * np.abs(ogx) + 1e-5 * np.abs(ogx).max())


def test_central_differences_on_the_gpu(sb, diff_case):
    c = diff_case
    p = _params(sb, c["prm"])
    _, gl, gs, _ = _gpu_grad(sb, p, c["xyz"], c["lab"], c["held"], c["held_lab"])

    def ll_at(**kw):
        q = _params(sb, c["prm"], **kw)
        with sb.Map(q) as m:
            m.insert_training(c["xyz"], c["lab"])
            return m.heldout_loglik(c["held"], c["held_lab"])

    l0, s0 = c["prm"]["length_scale"], c["prm"]["sigma0"]
    h = 1e-3
    fd_s = (ll_at(sigma0=s0 * (1 + h)) - ll_at(sigma0=s0 * (1 - h))) / (2 * h * s0)
    fd_l = (ll_at(length_scale=l0 * (1 + h)) - ll_at(length_scale=l0 * (1 - h))) / (2 * h * l0)
    assert abs(fd_s - gs) <= 1e-3 * abs(gs), (fd_s, gs)
    assert abs(fd_l - gl) <= 1e-3 * abs(gl), (fd_l, gl)


def test_upstream_gradient_sigma0_identity_and_stateless_forms(sb, diff_case):
    """For any upstream G at the map's voxels, dL/dsigma0 = sum G (alpha - alpha0)/sigma0
    (alpha - alpha0 is linear in sigma0); the stateless and map forms agree."""
    c = diff_case
    p = _params(sb, c["prm"])
    xyzl = np.concatenate([c["xyz"], c["lab"][:, None].astype(np.float32)], 1)
    keys, alpha = sb.forward_alpha(p, xyzl)
    rng = np.random.default_rng(5)
    G = rng.standard_normal(alpha.shape).astype(np.float32)
    gl, gs, gx = sb.grad(p, xyzl, keys, G)
    expect = float(np.sum(G.astype(np.float64) * (alpha.astype(np.float64) - c["prm"]["alpha0"]))) / c["prm"]["sigma0"]
    assert abs(gs - expect) <= 1e-4 * np.sum(np.abs(G) * (alpha - c["prm"]["alpha0"])) / c["prm"]["sigma0"]
    with sb.Map(p) as m:
        m.insert_training(c["xyz"], c["lab"])
        k2, a2, _ = m.export()
        np.testing.assert_array_equal(k2, keys)
        np.testing.assert_allclose(a2, alpha, rtol=1e-5)  # reductions in another order
        m.grad_clear()
        assert m.grad_add_alpha(keys, G) == 0
        gl2, gs2, gx2 = m.backward(xyzl)
    assert abs(gl2 - gl) <= 1e-6 * abs(gl) and abs(gs2 - gs) <= 1e-6 * abs(gs)
    np.testing.assert_allclose(gx2, gx, rtol=1e-5, atol=1e-6 * np.abs(gx).max())
    # a key no block holds is counted, not an error
    with sb.Map(p) as m:
        m.insert_training(c["xyz"], c["lab"])
        far = np.array([[100000, 100000, 100000]], np.int64)
        assert m.grad_add_alpha(far, np.ones((1, alpha.shape[1]), np.float32)) == 1


def test_autograd_functions(sb, diff_case):
    import torch
    from paper_1909_04631_gb300 import autograd as ag
    c = diff_case
    p = _params(sb, c["prm"])
    xyz = torch.from_numpy(c["xyz"]).cuda().requires_grad_(True)
    lab = torch.from_numpy(c["lab"]).cuda()
    l = torch.tensor(c["prm"]["length_scale"], dtype=torch.float32, requires_grad=True)
    s = torch.tensor(c["prm"]["sigma0"], dtype=torch.float32, requires_grad=True)
    held = torch.from_numpy(c["held"]).cuda()
    held_lab = torch.from_numpy(c["held_lab"].astype(np.int32)).cuda()
    ll = ag.heldout_loglik(xyz, lab, l, s, held, held_lab, p)
    (2.0 * ll).backward()
    ll0, gl, gs, gx = _gpu_grad(sb, p, c["xyz"], c["lab"], c["held"], c["held_lab"])
    assert abs(float(ll) - ll0) <= 1e-6 * abs(ll0)  # two forward runs: reductions in another order
    assert abs(float(l.grad) - 2 * gl) <= 1e-5 * abs(2 * gl)
    assert abs(float(s.grad) - 2 * gs) <= 1e-5 * abs(2 * gs)
    np.testing.assert_allclose(xyz.grad.cpu().numpy(), 2 * gx, rtol=1e-4, atol=1e-6 * np.abs(gx).max())
    # (keys, alpha) form: d(sum w * alpha)/dsigma0 = sum w (alpha - alpha0) / sigma0
    s2 = torch.tensor(c["prm"]["sigma0"], dtype=torch.float32, requires_grad=True)
    keys, alpha = ag.sbki_alpha(xyz.detach(), lab, l.detach(), s2, p)
    w = torch.linspace(-1.0, 1.0, alpha.numel(), device=alpha.device).reshape(alpha.shape)
    (w * alpha).sum().backward()
    expect = float(((w.double() * (alpha.double() - c["prm"]["alpha0"])).sum()) / c["prm"]["sigma0"])
    assert abs(float(s2.grad) - expect) <= 1e-4 * float((w.abs().double() * alpha.double()).sum())


def test_gradient_with_class_scales_matches_oracle(sb, orc, diff_case):
    """Per-class kernel scales (class k's kernel sigma0 s_k f): LL, dLL/dl,
    dLL/dsigma0, dLL/dxyz and dLL/ds_k against the oracle."""
    c = diff_case
    K1 = c["prm"]["num_classes"] + 1
    scale = [0.6 + 0.15 * k for k in range(K1)]
    p = _params(sb, c["prm"])
    sb.set_param(p, "sigma0_scale", scale)
    xyzl = np.concatenate([c["xyz"], c["lab"][:, None].astype(np.float32)], 1)
    with sb.Map(p) as m:
        m.insert_training(c["xyz"], c["lab"])
        m.grad_clear()
        ll = m.heldout_loglik(c["held"], c["held_lab"], grad=True)
        gl, gs, gx = m.backward(xyzl)
        gsc = m.backward_scales(xyzl)
    op = orc.params(**dict(c["prm"], sigma0_scale=scale))
    x64 = c["xyz"].astype(np.float64)
    oll, ogl, ogs, ogx = orc.heldout_grad(op, x64, c["lab"], c["held"], c["held_lab"])
    _, ogsc = orc.heldout_grad_scale(op, x64, c["lab"], c["held"], c["held_lab"])
    assert abs(ll - oll) <= 1e-5 * abs(oll)
    assert abs(gl - ogl) <= 1e-4 * abs(ogl) and abs(gs - ogs) <= 1e-4 * abs(ogs)
    err = np.abs(gx.astype(np.float64) - ogx)
    assert np.linalg.norm(err) <= 1e-4 * np.linalg.norm(ogx)
    used = np.abs(ogsc) > 0
    assert used.sum() >= 3
    np.testing.assert_allclose(gsc[used], ogsc[used], rtol=1e-4)
    assert np.all(gsc[~used] == 0)
    # the scaling identity holds on the GPU too
    assert float(np.dot(scale, gsc)) == pytest.approx(c["prm"]["sigma0"] * gs, rel=1e-6)
