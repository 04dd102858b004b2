"""Learned warm start for the GMM fit (an addition to the paper's method).

The paper starts every reconstruction from random Gaussians (Sec. 4.1: means
N(0, 0.075^2), scales 0.0075, amplitudes 1 / (2N)) and optimizes them with Adam.  This
module learns a better starting point:

1. ``coarse_volume``: the particle images, multiplied by their CTF (the adjoint of the CTF
   step, App. A.2 Eq. 14), are backprojected into a Dv^3 volume (gs_backproject, Dv = 32),
   and the total amplitude is estimated from the images' DC terms (gs_mass_estimate).
2. ``draw_seeds``: K seeds are drawn from the positive part of that volume
   (gs_seed_sample) and described by 32 features each (gs_seed_features).
3. ``PointMLP`` (3 layers, width 128, BF16 operands with FP32 accumulation; training and
   inference run in the library's own kernels) maps each seed's features to 10 numbers:
   an offset of the centre, a log-Cholesky covariance and a relative amplitude, which
   gs_decode_seeds turns into one raw Gaussian per seed.
4. Training pairs come from the plain method itself: ``build_dataset`` simulates
   random-walk-chain molecules, fits each with the plain method from random init
   (``fit``), and labels every seed with the moment-matched merge of the fitted Gaussians
   nearest to it (gs_merge_labels): a coarse-graining of the fitted mixture that keeps its
   mass and its first two moments locally.
5. ``initial_theta`` returns the learned start, or the paper's random init when no network
   is given (the fallback); ``steps_to_target`` judges a start by the number of Adam steps
   its fit needs to come within 1% of the loss that the random-init fit converges to.

The simulated molecules have unit total amplitude: the paper's random init (total
amplitude 1/2) assumes images on that scale, and a different scale would only measure how
long Adam takes to fix a unit mismatch.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from . import synth
from . import volume
from .splat import Splatter

DIN, HIDDEN, DOUT = 32, 128, 10
DV = 32


# --------------------------------------------------------------------------------- MLP
class PointMLP:
    """Parameters, Adam state and buffers of the point-MLP; every step runs in libgs."""

    def __init__(self, hidden=HIDDEN, din=DIN, dout=DOUT, seed=0, device="cuda"):
        self.dims = (int(din), int(hidden), int(dout))
        self.device = torch.device(device)
        n = L.gs_mlp_param_count(*self.dims)
        rng = np.random.default_rng(seed)
        p = np.zeros(n, dtype=np.float32)
        off = 0
        for fan_out, fan_in, gain in ((hidden, din, 2.0), (hidden, hidden, 2.0), (dout, hidden, 0.1)):
            w = rng.standard_normal(fan_out * fan_in) * math.sqrt(gain / fan_in)
            p[off:off + w.size] = w
            off += w.size + fan_out  # bias stays zero
        assert off == n
        self.params = torch.from_numpy(p).to(self.device)
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self._n = 0

    def _buffers(self, n):
        if n > self._n:
            din, hidden, dout = self.dims
            self._acts = torch.empty(n * 4 * hidden, dtype=torch.float32, device=self.device)
            self._scratch = torch.empty(n * 2 * hidden, dtype=torch.float32, device=self.device)
            self._Y = torch.empty((n, dout), dtype=torch.float32, device=self.device)
            self._dY = torch.empty((n, dout), dtype=torch.float32, device=self.device)
            self._n = n
        return self._acts, self._scratch, self._Y[:n], self._dY[:n]

    def predict(self, X, chunk=1 << 16):
        """Y[n, dout] for features X[n, din] (device)."""
        n = X.shape[0]
        out = torch.empty((n, self.dims[2]), dtype=torch.float32, device=self.device)
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            acts, _, Y, _ = self._buffers(b - a)
            L.gs_mlp_forward(self.params, self.dims, X[a:b], acts, out[a:b])
        return out

    def train_step(self, X, T, idx, lr):
        """One Adam step on the rows idx (int32, device) of the dataset (X, T).  Returns the
        minibatch loss (device, mean squared error)."""
        n = idx.numel()
        acts, scratch, Y, dY = self._buffers(n)
        self.grad.zero_()
        self.loss.zero_()
        L.gs_mlp_forward(self.params, self.dims, X, acts, Y, idx=idx)
        L.gs_mse(Y, T, self.loss, dY, idx=idx)
        L.gs_mlp_backward(self.params, self.dims, X, acts, dY, self.grad, scratch, idx=idx)
        self.t += 1
        L.gs_step(self.params, self.grad, self.m, self.v, self.t, lr=lr)
        return self.loss

    def evaluate(self, X, T, chunk=1 << 16):
        """Mean squared error over a whole set (device scalar)."""
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        n = X.shape[0]
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            acts, _, Y, _ = self._buffers(b - a)
            L.gs_mlp_forward(self.params, self.dims, X[a:b], acts, Y)
            L.gs_mse(Y, T[a:b], loss, None, scale=1.0 / (n * self.dims[2]))
        return loss

    def state(self):
        return {"dims": self.dims, "params": self.params.detach().cpu().numpy()}

    @classmethod
    def from_state(cls, st, device="cuda"):
        din, hidden, dout = (int(x) for x in st["dims"])
        net = cls(hidden, din, dout, device=device)
        net.params.copy_(torch.from_numpy(np.asarray(st["params"], dtype=np.float32)))
        return net

    @classmethod
    def load(cls, path, device="cuda"):
        with np.load(path) as f:
            return cls.from_state({"dims": f["dims"], "params": f["params"]}, device)


def load_pretrained(device="cuda"):
    """The network trained by ``python -m paper_2508_04929_b300.warmstart --molecules 2000``
    (D = 128, N 5k-50k, 39M labelled seeds), shipped with the package."""
    import os
    return PointMLP.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "pointmlp_d128.npz"),
                         device)


# --------------------------------------------------------------------------------- data
@dataclass
class Molecule:
    theta_gt: torch.Tensor  # [N, 11] ground truth (raw)
    W: torch.Tensor         # [P, 9]
    ctf: torch.Tensor       # [P, 5]
    Y: torch.Tensor         # [P, D, D] observed images
    D: int

    @property
    def N(self):
        return self.theta_gt.shape[0]


def unit_mass(theta):
    """Rescale the amplitudes of raw theta so that sum A = 1 (numpy, float32)."""
    th = np.asarray(theta, dtype=np.float64).copy()
    A = np.log1p(np.exp(th[:, 10]))
    th[:, 10] = synth.inv_softplus(A / A.sum())
    return th.astype(np.float32)


def simulate(sp: Splatter, N, P, rng, snr=0.1, device="cuda", seed=0):
    """A random-walk-chain molecule of N Gaussians (unit total amplitude) and P noisy
    particle images (uniform poses, CTF as in synth.random_ctf, white noise at ``snr``)."""
    D, B = sp.D, sp.B
    theta = torch.from_numpy(unit_mass(synth.chain_gaussians(N, D, rng))).to(device)
    W = torch.from_numpy(synth.random_poses(P, rng).reshape(P, 9)).to(device)
    ctf = torch.from_numpy(synth.random_ctf(P, rng)).to(device)
    clean = torch.empty((P, D, D), dtype=torch.float32, device=device)
    for a in range(0, P, B):
        sp.forward(theta, W[a:a + B], ctf[a:a + B], grow=True)
        clean[a:a + B].copy_(sp.X)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    sigma = torch.sqrt(clean.var() / snr)
    Y = clean + sigma * torch.randn(clean.shape, generator=gen, device=device)
    return Molecule(theta, W, ctf, Y, D)


class _PairGuard:
    """Keeps the pair buffer of a Splatter ahead of the need without a host sync per step:
    every ``every`` steps the last count is read and the buffer grown to twice that if it
    is more than 70% full."""

    def __init__(self, sp: Splatter, every=20):
        self.sp, self.every, self.k = sp, every, 0

    def __call__(self):
        self.k += 1
        if self.k % self.every == 1:
            need = int(self.sp.n_pairs.item()) & 0xFFFFFFFF
            if need > 0.7 * self.sp.pairs.numel():
                self.sp.pairs = torch.empty(2 * need + 4096, dtype=torch.int32, device=self.sp.device)


def eval_loss(sp: Splatter, theta, mol: Molecule, eval_idx):
    """Sum of the per-image losses over the evaluation particles (device scalar)."""
    tot = torch.zeros((), dtype=torch.float32, device=theta.device)
    B = sp.B
    for a in range(0, eval_idx.numel(), B):
        idx = eval_idx[a:a + B]
        sp.forward(theta, mol.W[idx], mol.ctf[idx], grow=True)
        sp.loss_grad(sp.X, mol.Y[idx])
        tot += sp.loss[:B].sum()
    return tot


def eval_schedule(steps, every=25, fine_until=100, fine_every=5):
    """Evaluation steps: every ``fine_every`` up to ``fine_until``, then every ``every``."""
    s = set(range(0, min(fine_until, steps) + 1, fine_every)) | set(range(0, steps + 1, every)) | {steps}
    return sorted(s)


def fit(sp: Splatter, theta0, mol: Molecule, steps, lr=1e-3, eval_every=0, eval_idx=None, train_idx=None,
        seed=0, eval_at=None, snapshot_at=(), snapshots=None):
    """The plain method: Adam (one learning rate for all parameters, Sec. 4.1) on the
    summed squared error of minibatches of sp.B particles.  Returns (theta, steps, losses)
    with the evaluation loss recorded at the steps ``eval_at`` (or every ``eval_every``
    steps, and at 0 and the end)."""
    if eval_at is None and eval_every:
        eval_at = sorted(set(range(0, steps + 1, eval_every)) | {steps})
    eval_at = set(eval_at or ())
    dev = theta0.device
    theta = theta0.clone()
    dtheta = torch.zeros_like(theta)
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    t_dev = torch.zeros(1, dtype=torch.int32, device=dev)
    P = mol.W.shape[0]
    if train_idx is None:
        train_idx = torch.arange(P, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    order = train_idx[torch.randperm(train_idx.numel(), generator=gen, device=dev)]
    guard = _PairGuard(sp)
    rec_s, rec_l = [], []
    B = sp.B
    pos = 0
    snap = set(snapshot_at)
    for step in range(steps + 1):
        if step in snap and snapshots is not None:
            snapshots[step] = theta.clone()
        if step in eval_at:
            rec_s.append(step)
            rec_l.append(eval_loss(sp, theta, mol, eval_idx))
        if step == steps:
            break
        if pos + B > order.numel():
            order = train_idx[torch.randperm(train_idx.numel(), generator=gen, device=dev)]
            pos = 0
        idx = order[pos:pos + B]
        pos += B
        dtheta.zero_()
        sp.forward_backward(theta, mol.W[idx], mol.ctf[idx], mol.Y[idx], dtheta, grow=False)
        guard()
        L.gs_step_counted(theta, dtheta, m, v, t_dev, lr=lr)
    losses = [float(x) for x in torch.stack(rec_l).cpu()] if rec_l else []
    return theta, rec_s, losses


def coarse_volume(sp: Splatter, mol: Molecule, Dv=DV, idx=None):
    """(vol[Dv, Dv, Dv], mass[1]) from the particles idx (default all): backprojection of
    the CTF-multiplied images and the DC-term mass estimate."""
    dev = mol.Y.device
    if idx is None:
        idx = torch.arange(mol.W.shape[0], device=dev)
    B = sp.B
    n = (idx.numel() // B) * B
    idx = idx[:n]
    Yc = torch.empty((n, sp.D, sp.D), dtype=torch.float32, device=dev)
    for a in range(0, n, B):
        j = idx[a:a + B]
        sp.apply_ctf(mol.Y[j].contiguous(), mol.ctf[j].contiguous(), Yc[a:a + B])
    vol = torch.empty((Dv, Dv, Dv), dtype=torch.float32, device=dev)
    W = mol.W[idx].contiguous()
    L.gs_backproject(Yc, W, Dv, vol)
    mass = torch.empty(1, dtype=torch.float32, device=dev)
    scratch = torch.empty(2, dtype=torch.float64, device=dev)
    L.gs_mass_estimate(mol.Y[idx].contiguous(), mol.ctf[idx].contiguous(), scratch, mass)
    return vol, mass


def draw_seeds(vol, K, rng):
    """(pos[K, 3], vmax[1], features[K, 32]) of K seeds drawn from vol (uniforms from rng)."""
    dev = vol.device
    Dv = vol.shape[-1]
    u = torch.from_numpy(rng.random((K, 4), dtype=np.float32)).to(dev)
    cdf = torch.empty(Dv ** 3, dtype=torch.int64, device=dev)
    vmax = torch.empty(1, dtype=torch.float32, device=dev)
    pos = torch.empty((K, 3), dtype=torch.float32, device=dev)
    L.gs_seed_sample(vol, u, cdf, vmax, pos)
    feats = torch.empty((K, DIN), dtype=torch.float32, device=dev)
    L.gs_seed_features(vol, vmax, pos, feats)
    return pos, vmax, feats


def random_theta(N, rng, device="cuda"):
    """The paper's random initialization (Sec. 4.1)."""
    return torch.from_numpy(synth.paper_init(N, rng)).to(device)


def seed_theta(pos, mass, Dv=DV):
    """Warm start without the network: a Gaussian of isotropic scale dv/2 and amplitude
    M / K at every seed (no offset, log-scales log 1/2, relative mass 1)."""
    K = pos.shape[0]
    pred = torch.zeros((K, DOUT), dtype=torch.float32, device=pos.device)
    pred[:, 3:6] = math.log(0.5)
    pred[:, 9] = 1.0
    theta = torch.empty((K, 11), dtype=torch.float32, device=pos.device)
    L.gs_decode_seeds(pos, pred, Dv, mass, theta)
    return theta


def initial_theta(sp: Splatter, mol: Molecule, N, rng, net: PointMLP | None = None, Dv=DV, idx=None):
    """Starting Gaussians for a fit of N Gaussians: the learned warm start when a network
    is given, else the paper's random init."""
    if net is None:
        return random_theta(N, rng, mol.Y.device)
    vol, mass = coarse_volume(sp, mol, Dv, idx)
    pos, vmax, feats = draw_seeds(vol, N, rng)
    pred = net.predict(feats)
    theta = torch.empty((N, 11), dtype=torch.float32, device=pos.device)
    L.gs_decode_seeds(pos, pred, Dv, mass, theta)
    return theta


# --------------------------------------------------------------------------------- dataset
@dataclass
class Dataset:
    X: torch.Tensor       # [M, 32] features
    T: torch.Tensor       # [M, 10] labels
    owner: torch.Tensor   # [M] molecule index (int32)
    info: list


def label_molecule(sp: Splatter, mol: Molecule, theta_fit, rng, Dv=DV):
    """(features, labels) of N seeds of one molecule against its fitted GMM."""
    vol, mass = coarse_volume(sp, mol, Dv)
    K = theta_fit.shape[0]
    pos, vmax, feats = draw_seeds(vol, K, rng)
    labels = torch.empty((K, DOUT), dtype=torch.float32, device=pos.device)
    L.gs_merge_labels(pos, theta_fit.contiguous(), Dv, mass, labels)
    return feats, labels


def build_dataset(n_molecules, D=128, N_range=(5000, 50000), P=256, batch=32, fit_steps=600, lr=3e-3, seed=0,
                  device="cuda", log=None):
    """Simulate molecules, fit each with the plain method from random init and label its
    seeds.  Returns a Dataset (device tensors)."""
    rng = np.random.default_rng(seed)
    Ns = np.exp(rng.uniform(math.log(N_range[0]), math.log(N_range[1]), n_molecules)).astype(int)
    sp = Splatter(D, int(Ns.max()), batch, tile=8, chunk=128, device=device)
    Xs, Ts, Os, info = [], [], [], []
    t0 = time.time()
    for i, N in enumerate(Ns):
        mrng = np.random.default_rng([seed, i])
        mol = simulate(sp, int(N), P, mrng, device=device, seed=seed * 100003 + i)
        theta, _, _ = fit(sp, random_theta(int(N), mrng, device), mol, fit_steps, lr=lr, seed=i)
        feats, labels = label_molecule(sp, mol, theta, mrng)
        Xs.append(feats)
        Ts.append(labels)
        Os.append(torch.full((int(N),), i, dtype=torch.int32, device=device))
        info.append({"N": int(N)})
        if log and (i + 1) % max(1, n_molecules // 20) == 0:
            log(f"molecule {i + 1}/{n_molecules} N={N} ({time.time() - t0:.1f}s)")
    sp.close()
    return Dataset(torch.cat(Xs), torch.cat(Ts), torch.cat(Os), info)


def train(net: PointMLP, data: Dataset, epochs=20, batch=4096, lr=1e-3, val_frac=0.1, seed=0, log=None):
    """Adam on minibatches of seeds with a cosine learning-rate decay; the last
    ``val_frac`` of the molecules are held out.  Returns (train curve, validation loss)."""
    dev = data.X.device
    n_mol = int(data.owner.max().item()) + 1
    cut = n_mol - max(1, int(round(val_frac * n_mol))) if n_mol > 1 else n_mol
    tr = torch.nonzero(data.owner < cut).flatten().to(torch.int32)
    va = torch.nonzero(data.owner >= cut).flatten()
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    steps_per_epoch = max(1, tr.numel() // batch)
    total = epochs * steps_per_epoch
    curve = []
    k = 0
    for ep in range(epochs):
        perm = tr[torch.randperm(tr.numel(), generator=gen, device=dev)]
        acc = torch.zeros((), device=dev)
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch].contiguous()
            lr_k = lr * 0.5 * (1.0 + math.cos(math.pi * k / total))
            acc += net.train_step(data.X, data.T, idx, lr_k)[0]
            k += 1
        curve.append(float(acc) / steps_per_epoch)
        if log:
            log(f"epoch {ep + 1}/{epochs} train mse {curve[-1]:.4f}")
    val = float(net.evaluate(data.X[va], data.T[va])) if va.numel() else float("nan")
    return curve, val


# --------------------------------------------------------------------------------- judging
def steps_to_target(steps, losses, target):
    """First recorded step whose loss is at most ``target`` (None if never)."""
    for s, l in zip(steps, losses):
        if l <= target:
            return int(s)
    return None


def compare_starts(sp: Splatter, mol: Molecule, net: PointMLP, rng, steps=1500, eval_every=25, lr=3e-3,
                   n_eval=64, eval_at=None, fsc_at=(), apix=1.5):
    """Fits of one molecule from the random init, from bare seeds and from the learned
    start.  The target is 1.01 x the loss the random-init fit converges to, taken as the
    lowest evaluation loss of its run (the fit of a finite particle set overfits after
    that point).  Returns a dict of curves and steps-to-target."""
    dev = mol.Y.device
    P = mol.W.shape[0]
    eval_idx = torch.arange(P - n_eval, P, device=dev)
    train_idx = torch.arange(0, P - n_eval, device=dev)
    N = mol.N
    out = {}
    vol, mass = coarse_volume(sp, mol, idx=train_idx)
    starts = {
        "random": random_theta(N, rng, dev),
        "seeds": seed_theta(draw_seeds(vol, N, rng)[0], mass),
        "learned": initial_theta(sp, mol, N, rng, net, idx=train_idx),
    }
    vol_gt = volume.voxelize(mol.theta_gt, sp.D) if fsc_at else None
    for name, th0 in starts.items():
        snaps = {}
        _, s, l = fit(sp, th0, mol, steps, lr=lr, eval_every=eval_every, eval_idx=eval_idx, train_idx=train_idx,
                      eval_at=eval_at, snapshot_at=fsc_at, snapshots=snaps)
        out[name] = {"steps": s, "loss": l}
        if fsc_at:
            # the fitted mixture against the ground truth: FSC 0.5 resolution (Angstrom) per step
            out[name]["res_fsc05"] = {int(k): volume.resolution(volume.fsc(volume.voxelize(v, sp.D), vol_gt).cpu(),
                                                                apix, 0.5) for k, v in snaps.items()}
    conv = float(np.min(out["random"]["loss"]))
    target = 1.01 * conv
    for name in starts:
        out[name]["steps_to_target"] = steps_to_target(out[name]["steps"], out[name]["loss"], target)
    out["target"] = target
    out["converged"] = conv
    return out


# --------------------------------------------------------------------------------- experiment
def _timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def main(argv=None):
    """Build the training set from plain fits of simulated molecules, train the network and
    judge it on held-out molecules; prints one JSON summary line."""
    ap = argparse.ArgumentParser(description="learned warm start: train and judge")
    ap.add_argument("--molecules", type=int, default=2000)
    ap.add_argument("--D", type=int, default=128)
    ap.add_argument("--n-min", type=int, default=5000)
    ap.add_argument("--n-max", type=int, default=50000)
    ap.add_argument("--particles", type=int, default=512)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--fit-steps", type=int, default=1000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--eval-molecules", type=int, default=8)
    ap.add_argument("--eval-steps", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None, help="write the full result (JSON) here")
    ap.add_argument("--save-net", default=None, help="write the trained network (npz) here")
    ap.add_argument("--net", default=None,
                    help="evaluate this trained network (npz; 'pretrained' for the shipped one) instead of building a "
                         "dataset and training")
    ap.add_argument("--fsc-at", default="0,25,100,400",
                    help="steps at which the fits are compared with the ground truth by FSC")
    a = ap.parse_args(argv)
    fsc_at = tuple(int(x) for x in a.fsc_at.split(",") if x.strip())
    dev = "cuda"

    def log(msg):
        print(msg, file=sys.stderr, flush=True)

    if a.net:
        net = load_pretrained(dev) if a.net == "pretrained" else PointMLP.load(a.net, dev)
        curve, val, t_data, t_train, samples = [], float("nan"), 0.0, 0.0, 0
    else:
        data, t_data = _timed(lambda: build_dataset(a.molecules, D=a.D, N_range=(a.n_min, a.n_max), P=a.particles,
                                                    batch=a.batch, fit_steps=a.fit_steps, lr=a.lr, seed=a.seed,
                                                    device=dev, log=log))
        log(f"dataset: {data.X.shape[0]} seeds from {a.molecules} molecules in {t_data:.1f}s")
        net = PointMLP(seed=a.seed, device=dev)
        (curve, val), t_train = _timed(lambda: train(net, data, epochs=a.epochs, lr=2e-3, seed=a.seed, log=log))
        log(f"trained {a.epochs} epochs in {t_train:.1f}s, validation mse {val:.4f}")
        if a.save_net:
            np.savez(a.save_net, dims=np.asarray(net.dims), params=net.state()["params"])
        samples = data.X.shape[0]
        del data

    rng = np.random.default_rng([a.seed, 7919])
    Ns = np.exp(rng.uniform(math.log(a.n_min), math.log(a.n_max), a.eval_molecules)).astype(int)
    sp = Splatter(a.D, int(Ns.max()), a.batch, tile=8, chunk=128, device=dev)
    sched = eval_schedule(a.eval_steps)
    rows = []
    for i, N in enumerate(Ns):
        mrng = np.random.default_rng([a.seed, 104729, i])
        mol = simulate(sp, int(N), a.particles, mrng, device=dev, seed=10 ** 6 + i)
        res = compare_starts(sp, mol, net, mrng, steps=a.eval_steps, lr=a.lr, eval_at=sched, fsc_at=fsc_at)
        tr = torch.arange(0, a.particles - 64, device=dev)
        _, t_warm = _timed(lambda: initial_theta(sp, mol, int(N), mrng, net, idx=tr))
        _, t_steps = _timed(lambda: fit(sp, random_theta(int(N), mrng, dev), mol, 100, lr=a.lr, train_idx=tr))
        row = {"N": int(N), "target": res["target"], "warm_start_ms": 1e3 * t_warm, "adam_step_ms": 10.0 * t_steps}
        for k in ("random", "seeds", "learned"):
            row[k] = {"steps_to_target": res[k]["steps_to_target"], "loss0": res[k]["loss"][0],
                      "best": float(np.min(res[k]["loss"])), "steps": res[k]["steps"], "loss": res[k]["loss"],
                      "res_fsc05": res[k].get("res_fsc05", {})}
        rows.append(row)
        log(f"molecule N={N}: steps to target random {row['random']['steps_to_target']} seeds "
            f"{row['seeds']['steps_to_target']} learned {row['learned']['steps_to_target']}; FSC-0.5 resolution (A) "
            f"by step: " + "; ".join(f"{k} {row[k]['res_fsc05']}" for k in ("random", "seeds", "learned")))
    sp.close()

    def agg(k):
        v = [r[k]["steps_to_target"] for r in rows]
        ok = [x for x in v if x is not None]
        return {"median": float(np.median(ok)) if ok else None, "reached": len(ok), "of": len(v)}

    training = ({"network": a.net} if a.net else
                {"molecules": a.molecules, "fit_steps": a.fit_steps, "training_seeds": int(samples),
                 "dataset_s": round(t_data, 1), "train_s": round(t_train, 1), "val_mse": val})
    summary = {
        "experiment": "learned warm start", "D": a.D, "N_range": [a.n_min, a.n_max], "particles": a.particles,
        "lr": a.lr, "eval_molecules": a.eval_molecules, **training,
        "steps_to_target": {k: agg(k) for k in ("random", "seeds", "learned")},
        "learned_best_below_random_best": sum(r["learned"]["best"] < r["random"]["best"] for r in rows),
        "fsc05_resolution_median_A": {k: {st: float(np.median([r[k]["res_fsc05"][st] for r in rows]))
                                          for st in fsc_at} for k in ("random", "seeds", "learned")},
        "warm_start_ms_median": float(np.median([r["warm_start_ms"] for r in rows])),
        "adam_step_ms_median": float(np.median([r["adam_step_ms"] for r in rows])),
    }
    if a.out:
        with open(a.out, "w") as f:
            json.dump({"summary": summary, "molecules": rows, "train_curve": curve}, f)
    print(json.dumps(summary))
    return summary


if __name__ == "__main__":
    main()
