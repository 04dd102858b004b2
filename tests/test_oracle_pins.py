"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: numerical quadrature,
library routines (SciPy rotations and densities, NumPy FFTs, torch.optim.Adam), closed
forms (Poisson summation, the Fourier transform of a Gaussian, the Fourier slice theorem,
CTF zeros), brute-force enumeration and central finite differences.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import minimize_scalar
from scipy.spatial.transform import Rotation
from scipy.stats import multivariate_normal

import oracle as O
from paper_2508_04929_b300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
F64 = np.float64


def _indep_gaussian(theta_row):
    """mu, Sigma (3-D, world frame) and A built with SciPy, independently of the oracle."""
    th = np.asarray(theta_row, dtype=F64)
    s = np.log1p(np.exp(th[3:6]))
    q = th[6:10] / np.linalg.norm(th[6:10])
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # SciPy is scalar-last
    return th[0:3].copy(), R @ np.diag(s * s) @ R.T, float(np.log1p(np.exp(th[10])))


def _rot64(rng, n=1):
    """Exactly orthogonal FP64 rotations (the closed forms below need W^-1 = W^T to FP64
    precision, which FP32-rounded poses do not give)."""
    return Rotation.random(n, random_state=int(rng.integers(1 << 31))).as_matrix()


def _iso(theta, s_px, D):
    th = theta.copy()
    th[:, 3:6] = synth.inv_softplus(np.repeat(np.asarray(s_px)[:, None] / D, 3, axis=1))
    return th


# ---------------------------------------------------------------------------------------
# Projection, normalization, coordinates
# ---------------------------------------------------------------------------------------
def test_splat_is_line_integral_of_3d_gaussian():
    """Sec. 3.3.3 Eqs. 7-8: the splat equals the line integral of the viewed 3-D normalized
    Gaussian (Eq. 4, Eq. 6) along z.  Brute-force z-quadrature, 1e-10 relative."""
    rng = synth.rng_for(11)
    worst = 0.0
    for _ in range(4):
        th = synth.random_gaussians(1, 32, rng).astype(F64)
        W = _rot64(rng)[0]
        mu, Sig, _ = _indep_gaussian(th[0])
        g = O.build_gaussians(th)
        md, Sd = O.viewing_transform(g["mu"], g["Sigma"], W)
        mt, St = O.projection(md, Sd)
        sz = math.sqrt((W @ Sig @ W.T)[2, 2])
        zc = (W @ mu)[2]
        for _k in range(3):
            r = mt[0] + rng.normal(scale=1.5 * math.sqrt(St[0][0, 0]), size=2)
            val = O.splat(r, mt[0], St[0])
            f = lambda z: multivariate_normal.pdf(W.T @ np.array([r[0], r[1], z]), mean=mu, cov=Sig)
            logf = lambda z: -multivariate_normal.logpdf(W.T @ np.array([r[0], r[1], z]), mean=mu, cov=Sig)
            # the integrand along the beam peaks away from zc and is much narrower than
            # sz; locate the peak numerically and integrate on both sides of it
            zpk = minimize_scalar(logf, bounds=(zc - 14 * sz, zc + 14 * sz), method="bounded",
                                  options={"xatol": 1e-12 * sz}).x
            ref = sum(quad(f, a, b, epsabs=0.0, epsrel=1e-13, limit=400)[0]
                      for a, b in ((zc - 14 * sz, zpk), (zpk, zc + 14 * sz)))
            worst = max(worst, abs(val - ref) / abs(ref))
    assert worst < 1e-10, worst


def test_mass_conservation_wide_gaussians():
    """Sec. 3.3.3: with the view-dependent normalization kept, each splat integrates to A,
    so sum_p Q(p) h^2 = sum A for Gaussians inside the box (sigma >= 1 px, 8-sigma support;
    the Poisson-summation error is ~2 exp(-2 pi^2) ~ 5e-9)."""
    rng = synth.rng_for(12)
    D = 96
    th = synth.random_gaussians(30, D, rng, centre_radius=0.2, scale_px=(1.0, 2.4)).astype(F64)
    W = synth.random_poses(1, rng)[0]
    Q = O.render_one(th, W, D, cutoff=8.0)
    h = 1.0 / D
    A = O.softplus(th[:, 10])
    assert abs(Q.sum() * h * h - A.sum()) / A.sum() < 1e-7


def test_mass_of_narrow_splat_follows_poisson_summation():
    """At sigma = 0.5 px the pixel sum of a splat deviates from A by the aliasing terms of
    the Poisson summation formula: prod_axes [1 + 2 sum_m exp(-2 pi^2 sigma^2 m^2)
    cos(2 pi m phi)], phi the sub-pixel offset of the centre (Eq. 13 pixel centres)."""
    rng = synth.rng_for(13)
    D = 32
    devs = []
    for _ in range(5):
        sx, sy = rng.uniform(0.45, 0.7, size=2)
        cx, cy = rng.uniform(-3, 3, size=2)
        th = np.zeros((1, 11))
        th[0, 0:3] = [cx / D, cy / D, 0.123]
        th[0, 3:6] = synth.inv_softplus(np.array([sx, sy, 0.9]) / D)
        th[0, 6:10] = [1, 0, 0, 0]
        th[0, 10] = synth.inv_softplus(1.0)
        Q = O.render_one(th, np.eye(3), D, cutoff=9.0)
        total = Q.sum() / (D * D)
        pred = 1.0
        for s_, c_ in ((sx, cx), (sy, cy)):
            m = np.arange(1, 6)
            pred *= 1.0 + 2.0 * np.sum(np.exp(-2 * math.pi ** 2 * s_ ** 2 * m ** 2) * np.cos(2 * math.pi * m * c_))
        assert abs(total - pred) < 1e-10, (total, pred)
        devs.append(abs(pred - 1.0))
    assert max(devs) > 5e-3  # the effect is real at this width


def test_isotropic_pose_invariance():
    """App. D.2 Eq. 22: with s_x = s_y = s_z the Gaussian is isotropic, so its splat is
    sigma^2 I for every rotation and pose, and two poses give the same image once the
    centres are moved accordingly."""
    rng = synth.rng_for(14)
    D = 32
    th = synth.random_gaussians(25, D, rng).astype(F64)
    th = _iso(th, rng.uniform(0.8, 2.5, size=25), D)
    W1, W2 = _rot64(rng, 2)
    th2 = th.copy()
    th2[:, 0:3] = th[:, 0:3] @ (W2.T @ W1).T  # mu' = W2^T W1 mu
    th2[:, 6:10] = synth.random_gaussians(25, D, rng)[:, 6:10]  # any rotation
    Q1 = O.render_one(th, W1, D, cutoff=40.0)
    Q2 = O.render_one(th2, W2, D, cutoff=40.0)
    assert np.max(np.abs(Q1 - Q2)) <= 1e-11 * np.max(np.abs(Q1))
    g = O.build_gaussians(th2)
    _, Sd = O.viewing_transform(g["mu"], g["Sigma"], W2)
    s = O.softplus(th2[:, 3])
    assert np.allclose(Sd[:, 0:2, 0:2], s[:, None, None] ** 2 * np.eye(2)[None], rtol=1e-12, atol=1e-15 * s.max() ** 2)


def test_pixel_origin_and_y_flip():
    """App. A.2 Eq. 13 and App. A.1 Fig. rasterization (b): the origin sits on pixel
    [floor(D/2), floor(D/2)] ([2, 2] for a 4 x 4 image), rows are y flipped, columns x."""
    rx, ry = O.pixel_centres(4)
    oi, oj = GOLDEN["fft_origin_4x4"]["value"]
    assert rx[oi, oj] == 0.0 and ry[oi, oj] == 0.0
    assert np.all(np.diff(rx, axis=1) > 0) and np.all(np.diff(ry, axis=0) < 0)
    for D in (31, 32):
        c = D // 2
        for a, b in ((3, -5), (-7, 2), (0, 0)):
            th = np.zeros((1, 11))
            th[0, 0:3] = [a / D, b / D, -0.2]
            th[0, 3:6] = synth.inv_softplus(np.full(3, 1.5 / D))
            th[0, 6:10] = [1, 0, 0, 0]
            th[0, 10] = 1.0
            Q = O.render_one(th, np.eye(3), D, cutoff=5.0)
            i, j = np.unravel_index(np.argmax(Q), Q.shape)
            assert (i, j) == (c - b, c + a)


def _centred_dft(Q):
    D = Q.shape[0]
    c = D // 2
    k = np.arange(-(D // 2), D - D // 2)
    n = np.arange(D) - c
    E = np.exp(-2j * math.pi * np.outer(k, n) / D)
    return E @ Q @ E.T, k


def test_fourier_slice_theorem_fixes_origin_and_pose():
    """App. A.1 Eq. 11 (Fourier slice theorem): the DFT of a rendered splat, taken about
    the Eq. 13 origin, equals the 3-D Gaussian's Fourier transform on the central slice
    W^T [kx, ky, 0] -- computed from the 3-D mu and Sigma, not from the 2 x 2 marginal."""
    rng = synth.rng_for(15)
    D = 96
    h = 1.0 / D
    for _ in range(3):
        th = synth.random_gaussians(1, D, rng, centre_radius=0.15, scale_px=(2.5, 3.0)).astype(F64)
        W = _rot64(rng)[0]
        Q = O.render_one(th, W, D, cutoff=9.0)
        S, k = _centred_dft(Q)
        mu, Sig, A = _indep_gaussian(th[0])
        KI, KJ = np.meshgrid(k, k, indexing="ij")
        kap = np.stack([KJ / (D * h), -KI / (D * h), 0 * KI], -1)  # row index is -y
        k3 = kap @ W  # W^T kappa, row-vector form
        pred = (A / h ** 2) * np.exp(-2 * math.pi ** 2 * np.einsum("...a,ab,...b->...", k3, Sig, k3)
                                     - 2j * math.pi * (k3 @ mu))
        err = np.max(np.abs(S - pred)) / np.max(np.abs(pred))
        assert err < 1e-10, err


def test_image_centred_origin_has_the_papers_phase_error():
    """Negative test, App. A.1 Fig. rasterization (b): sampling about the image centre
    (D-1)/2 instead of floor(D/2) is a half-pixel shift, which multiplies the spectrum by a
    phase of magnitude pi k / D (pi / 2 at Nyquist, k = D / 2)."""
    rng = synth.rng_for(16)
    D = 64
    h = 1.0 / D
    th = synth.random_gaussians(1, D, rng, centre_radius=0.1, scale_px=(2.5, 3.0)).astype(F64)
    W = _rot64(rng)[0]
    Q = O.render_one(th, W, D, cutoff=9.0)
    th2 = th.copy()
    th2[0, 0:3] += W.T @ np.array([-h / 2, h / 2, 0.0])  # what an image-centred raster samples
    Q2 = O.render_one(th2, W, D, cutoff=9.0)
    S, k = _centred_dft(Q)
    S2, _ = _centred_dft(Q2)
    c = D // 2
    kk = np.arange(1, D // 4)
    ph = np.angle(S2[c, c + kk] / S[c, c + kk])  # along k_x, k_y = 0
    assert np.allclose(np.abs(ph), math.pi * kk / D, atol=1e-9)
    nyq = math.pi * (D / 2) / D
    assert abs(nyq - GOLDEN["image_centred_phase_error_at_nyquist"]["value"]) < 1e-15


# ---------------------------------------------------------------------------------------
# Support rule and tile binning
# ---------------------------------------------------------------------------------------
def test_support_box_matches_fp64_definition_away_from_ties():
    """The FP32 box equals the box of the FP64 definition (ceil/floor of c -/+ k sqrt(Sigma)
    / h, built with SciPy) for every Gaussian whose FP64 bounds are not within 1e-3 px of an
    integer; catches a wrong axis, sign, index or scale in the FP32 decision path."""
    rng = synth.rng_for(17)
    D = 64
    th = synth.random_gaussians(800, D, rng)
    checked = 0
    for W in synth.random_poses(3, rng):
        x0, x1, y0, y1, bad = O.support_fp32(th, W, D)
        assert not bad.any()
        Wd = W.astype(F64)
        for n in range(th.shape[0]):
            mu, Sig, _ = _indep_gaussian(th[n])
            St = (Wd @ Sig @ Wd.T)[0:2, 0:2]
            m = Wd @ mu
            cx, cy = m[0] * D + D // 2, D // 2 - m[1] * D
            rx, ry = 3 * math.sqrt(St[0, 0]) * D, 3 * math.sqrt(St[1, 1]) * D
            bounds = (cx - rx, cx + rx, cy - ry, cy + ry)
            if min(abs(b - round(b)) for b in bounds) < 1e-3:
                continue
            ref = (max(math.ceil(bounds[0]), 0), min(math.floor(bounds[1]), D - 1),
                   max(math.ceil(bounds[2]), 0), min(math.floor(bounds[3]), D - 1))
            assert (x0[n], x1[n], y0[n], y1[n]) == ref
            checked += 1
    assert checked > 2300


def test_tile_pairs_match_brute_force_enumeration():
    """Algorithm 2 CreateTiles .. IdentifyTileRanges: the sorted (particle, tile, Gaussian)
    instances equal a brute-force pixel-by-pixel enumeration, for a box that is not a
    multiple of the tile (ragged last tile)."""
    rng = synth.rng_for(18)
    D, T = 40, 16
    th = synth.random_gaussians(60, D, rng)
    Ws = synth.random_poses(2, rng)
    pg, ranges = O.tile_pairs(th, Ws, D, T)
    nt = -(-D // T)
    expect = []
    for b in range(2):
        x0, x1, y0, y1, _ = O.support_fp32(th, Ws[b], D)
        for t in range(nt * nt):
            ty, tx = divmod(t, nt)
            for n in range(60):
                pix = [(i, j) for i in range(y0[n], y1[n] + 1) for j in range(x0[n], x1[n] + 1)]
                if any(i // T == ty and j // T == tx for i, j in pix):
                    expect.append((b, t, n))
    got = []
    for b in range(2):
        for t in range(nt * nt):
            s, e = ranges[b, t]
            got += [(b, t, int(g)) for g in pg[s:e]]
    assert got == expect
    assert ranges[-1, -1, 1] == len(pg)


@pytest.mark.parametrize("D,T", [(40, 8), (33, 16), (50, 32), (64, 8)])
def test_tile_counts_match_brute_force_enumeration(D, T):
    """tile_counts (the checker of the full-size GPU tests) equals, per (particle, tile), the
    number of Gaussians with a pixel of their support box in that tile, found by enumerating
    every box pixel; and equals the run lengths of tile_pairs.  Ragged D, boxes of several
    tiles, and boxes clipped at every image edge (centres out to 0.6 D)."""
    rng = synth.rng_for(19)
    th = synth.random_gaussians(150, D, rng, centre_radius=0.6, scale_px=(0.5, 6.0))
    Ws = synth.random_poses(3, rng)
    got = O.tile_counts(th, Ws, D, T)
    nt = -(-D // T)
    expect = np.zeros((3, nt * nt), dtype=np.int64)
    clipped = 0
    for b in range(3):
        x0, x1, y0, y1, _ = O.support_fp32(th, Ws[b], D)
        for n in range(150):
            tiles = {(i // T) * nt + (j // T) for i in range(y0[n], y1[n] + 1) for j in range(x0[n], x1[n] + 1)}
            for t in tiles:
                expect[b, t] += 1
            clipped += int(x0[n] == 0 or y0[n] == 0 or x1[n] == D - 1 or y1[n] == D - 1)
    assert clipped > 10 and expect.max() > 1
    assert np.array_equal(got, expect)
    _, ranges = O.tile_pairs(th, Ws, D, T)
    assert np.array_equal(got, (ranges[:, :, 1] - ranges[:, :, 0]).astype(np.int64))


def test_truncation_error_is_bounded_by_tail_mass():
    """The 3-sigma support only drops positive mass, at most the mass outside the box:
    P(|x| > 3 sigma_x) + P(|y| > 3 sigma_y) = 2 x 0.0027 per splat (plus sampling error)."""
    rng = synth.rng_for(19)
    D = 64
    th = synth.random_gaussians(80, D, rng, centre_radius=0.2, scale_px=(1.0, 3.0)).astype(F64)
    W = synth.random_poses(1, rng)[0]
    Q3 = O.render_one(th, W, D, cutoff=3.0)
    Qf = O.render_one(th, W, D, cutoff=12.0)
    assert np.min(Qf - Q3) >= -1e-12 * np.max(Qf)
    A = O.softplus(th[:, 10]).sum()
    lost = (Qf - Q3).sum() / D ** 2
    assert 0.0 < lost <= (2 * 0.0027 + 1e-3) * A


# ---------------------------------------------------------------------------------------
# CTF, DFT, loss
# ---------------------------------------------------------------------------------------
def test_electron_wavelength_300kv():
    """Relativistic electron wavelength at 300 kV: 0.019687 A (textbook value)."""
    assert abs(O.electron_wavelength(300.0) - 0.0196875) < 2e-7


def test_ctf_dc_value_and_zeros():
    """H_hat(0) = -w; with Cs = 0 the zeros sit where sin(chi + asin w) = 0, i.e.
    |k|^2 = (n pi - asin w) / (pi lambda df) -- a hand-derived closed form."""
    for w in (0.07, 0.1):
        assert abs(O.ctf_radial(0.0, 15000.0, 300.0, 2.7, w) + w) < 1e-15
        lam = O.electron_wavelength(300.0)
        for n in (1, 2, 5):
            k2 = (n * math.pi - math.asin(w)) / (math.pi * lam * 15000.0)
            assert abs(O.ctf_radial(k2, 15000.0, 300.0, 0.0, w)) < 1e-12
    H = O.ctf_image(33, 20000.0)
    assert np.allclose(H, H[(-np.arange(33)) % 33][:, (-np.arange(33)) % 33], atol=0)


def test_direct_dft_matches_numpy_fft():
    rng = synth.rng_for(20)
    for D in (8, 15):
        x = rng.standard_normal((D, D))
        assert np.allclose(O.dft2(x), np.fft.fft2(x), atol=1e-10)
        z = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
        assert np.allclose(O.idft2(z), np.fft.ifft2(z), atol=1e-12)


def test_ctf_operator_is_real_self_adjoint_and_shift_invariant():
    """H_hat is real and even, so X = F^-1(H F Q) is real, the operator equals its adjoint,
    and it commutes with the fftshift re-centring (the result does not depend on where the
    DFT puts the origin)."""
    rng = synth.rng_for(21)
    for D in (16, 17):
        H = O.ctf_image(D, 18000.0, apix=2.0)
        Q = rng.standard_normal((D, D))
        Y = rng.standard_normal((D, D))
        Z = O.idft2(H * O.dft2(Q))
        assert np.max(np.abs(Z.imag)) < 1e-12 * np.max(np.abs(Z.real))
        CQ = O.apply_ctf(Q, H)
        CtY = O.apply_ctf_adjoint(Y, H)
        assert abs(np.sum(CQ * Y) - np.sum(Q * CtY)) < 1e-10 * np.sqrt(np.sum(CQ ** 2) * np.sum(Y ** 2))
        assert np.allclose(O.apply_ctf(Y, H), CtY, atol=1e-12)
        assert np.allclose(O.apply_ctf(np.fft.ifftshift(Q), H), np.fft.ifftshift(CQ), atol=1e-12)
        # against NumPy's FFT
        ref = np.fft.ifft2(H * np.fft.fft2(Q)).real
        assert np.allclose(CQ, ref, atol=1e-12)


def test_loss_parseval_and_gradient():
    """Sec. 3.3.5 L = ||X - Y||^2: equals (1 / D^2) sum |F(X - Y)|^2 (Parseval); dL/dX by
    central differences."""
    rng = synth.rng_for(22)
    X = rng.standard_normal((2, 12, 12))
    Y = rng.standard_normal((2, 12, 12))
    L, G = O.loss(X, Y)
    spec = np.sum(np.abs(np.fft.fft2(X - Y)) ** 2, axis=(1, 2)) / 144
    assert np.allclose(L, spec, rtol=1e-13)
    e = 1e-6
    for (b, i, j) in ((0, 3, 4), (1, 11, 0)):
        Xp, Xm = X.copy(), X.copy()
        Xp[b, i, j] += e
        Xm[b, i, j] -= e
        fd = (O.loss(Xp, Y)[0][b] - O.loss(Xm, Y)[0][b]) / (2 * e)
        assert abs(fd - G[b, i, j]) < 1e-7
    Lm, Gm = O.loss(X, Y, reduction=1)
    assert np.allclose(Lm * 144, L) and np.allclose(Gm * 144, G)


# ---------------------------------------------------------------------------------------
# Backward by central finite differences (support frozen at the base point)
# ---------------------------------------------------------------------------------------
def _fd_setup(seed=23, N=200, D=32, B=2):
    rng = synth.rng_for(seed)
    th = synth.random_gaussians(N, D, rng).astype(F64)
    Ws = synth.random_poses(B, rng).astype(F64)
    ctf = synth.random_ctf(B, rng)
    Hs = [O.ctf_image(D, *[float(v) for v in ctf[b, [0, 1, 2, 3]]], apix=float(ctf[b, 4])) for b in range(B)]
    ref_th = synth.random_gaussians(N, D, rng).astype(F64)
    Y = np.stack([O.apply_ctf(O.render_one(ref_th, Ws[b], D), Hs[b]) for b in range(B)])
    Y = Y + 0.1 * rng.standard_normal(Y.shape) * Y.std()
    boxes = [O.support_fp32(th, Ws[b], D)[:4] for b in range(B)]
    return th, Ws, Hs, Y, boxes, D


def _analytic_grad(th, Ws, Hs, Y, boxes, D, transpose_mu=True):
    Q = np.stack([O.render_one(th, Ws[b], D, box=boxes[b]) for b in range(len(Ws))])
    X = np.stack([O.apply_ctf(Q[b], Hs[b]) for b in range(len(Ws))])
    _, dX = O.loss(X, Y)
    dQ = np.stack([O.apply_ctf_adjoint(dX[b], Hs[b]) for b in range(len(Ws))])
    return Q, O.backward(th, Ws, D, dQ, boxes=boxes)


def test_backward_matches_central_differences():
    """App. A.2 Eqs. 16-21 (+ the 3DGS chain for s, q and the softplus derivatives):
    the oracle gradient equals FP64 central differences (h = 1e-6) of the oracle loss at
    N = 200, D = 32, per parameter group, with the support frozen at the base point."""
    th, Ws, Hs, Y, boxes, D = _fd_setup()
    Q, g = _analytic_grad(th, Ws, Hs, Y, boxes, D)
    B = len(Ws)

    def splat_img(row, b, n):
        box = tuple(np.array([boxes[b][k][n]]) for k in range(4))
        return O.render_one(row[None], Ws[b], D, box=box)

    def L_of(Qs):
        return sum(np.sum((O.apply_ctf(Qs[b], Hs[b]) - Y[b]) ** 2) for b in range(B))

    base = [[splat_img(th[n], b, n) for n in range(th.shape[0])] for b in range(B)]
    e = 1e-6
    fd = np.zeros_like(g)
    for n in range(th.shape[0]):
        for p in range(11):
            vals = []
            for sgn in (1, -1):
                row = th[n].copy()
                row[p] += sgn * e
                Qs = [Q[b] - base[b][n] + splat_img(row, b, n) for b in range(B)]
                vals.append(L_of(Qs))
            fd[n, p] = (vals[0] - vals[1]) / (2 * e)
    for name, sl in (("mu", slice(0, 3)), ("s", slice(3, 6)), ("q", slice(6, 10)), ("A", slice(10, 11))):
        rel = np.linalg.norm(g[:, sl] - fd[:, sl]) / np.linalg.norm(fd[:, sl])
        assert rel < 1e-7, (name, rel)


def test_printed_W_in_mean_gradient_is_a_misprint():
    """App. A.2 Eq. 18 prints grad_mu = W [grad_mu_tilde; 0]; since mu_dot = W mu (Eq. 6)
    the chain rule gives W^T.  Central differences agree with W^T and not with W."""
    th, Ws, Hs, Y, boxes, D = _fd_setup(seed=24, N=6, D=24, B=1)
    Q, g = _analytic_grad(th, Ws, Hs, Y, boxes, D)
    W = Ws[0]

    def L_of(t):
        Qb = O.render_one(t, W, D, box=boxes[0])
        return np.sum((O.apply_ctf(Qb, Hs[0]) - Y[0]) ** 2)

    e = 1e-6
    fd = np.zeros((th.shape[0], 3))
    for n in range(th.shape[0]):
        for p in range(3):
            tp, tm = th.copy(), th.copy()
            tp[n, p] += e
            tm[n, p] -= e
            fd[n, p] = (L_of(tp) - L_of(tm)) / (2 * e)
    assert np.linalg.norm(g[:, 0:3] - fd) < 1e-6 * np.linalg.norm(fd)
    printed = g[:, 0:3] @ W.T @ W.T  # W (W W^T)... = W applied to grad_mu_tilde
    assert np.linalg.norm(printed - fd) > 1e-2 * np.linalg.norm(fd)


# ---------------------------------------------------------------------------------------
# Adam
# ---------------------------------------------------------------------------------------
def test_adam_matches_torch_and_first_step_closed_form():
    """Sec. 4.1: Adam with one learning rate.  Against torch.optim.Adam (CPU, FP64) over
    five steps, and the closed-form first step -lr sign(g) for |g| >> eps."""
    import torch
    rng = synth.rng_for(25)
    th = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(5)]
    p = torch.tensor(th.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    x = th.copy()
    for t, gr in enumerate(grads, start=1):
        opt.zero_grad()
        p.grad = torch.tensor(gr)
        opt.step()
        x, m, v = O.adam_step(x, gr, m, v, t)
    assert np.allclose(x, p.detach().numpy(), rtol=0, atol=1e-15)
    x1, _, _ = O.adam_step(th, grads[0], np.zeros(50), np.zeros(50), 1)
    assert np.allclose(x1 - th, -1e-3 * np.sign(grads[0]), atol=1e-10)


def test_paper_initialization_values():
    """Sec. 4.1: mean spread 0.9 E / 6 = 0.075, scale 0.0075, A = 1 / (2N)."""
    E = GOLDEN["E"]["value"]
    assert abs(0.9 * E / 6 - GOLDEN["init_mean_sigma"]["value"]) < 1e-15
    rng = synth.rng_for(26)
    th = synth.paper_init(20000, rng).astype(F64)
    assert abs(th[:, 0:3].std() - GOLDEN["init_mean_sigma"]["value"]) < 2e-3
    assert np.allclose(O.softplus(th[:, 3:6]), GOLDEN["init_scale"]["value"], rtol=1e-6)
    assert np.allclose(O.softplus(th[:, 10]) * 2 * 20000, GOLDEN["init_amplitude_times_2N"]["value"], rtol=1e-5)
