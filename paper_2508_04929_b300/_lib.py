"""ctypes binding of libgs.so (include/gs.h).  Argument marshalling only.

Every function here has the name of the C entry point it calls and takes torch tensors
(device memory) plus plain Python values; it passes their data pointers and the current
CUDA stream to the library and raises ``GsError`` on a non-zero return code.  There is no
fallback: if libgs.so is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs.so")

GS_OK, GS_EINVAL, GS_ENOSPC, GS_ECUDA = 0, 1, 2, 3
GS_STATUS_NONFINITE, GS_STATUS_OVERFLOW = 1, 2
RECORD_BYTES = 32

_ERR = {GS_EINVAL: "invalid argument", GS_ENOSPC: "buffer too small", GS_ECUDA: "CUDA/cuFFT failure"}


class GsError(RuntimeError):
    def __init__(self, name, rc):
        super().__init__(f"{name} failed: {_ERR.get(rc, rc)} (code {rc})")
        self.rc = rc


class GsConfig(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("E", ctypes.c_float), ("tile", ctypes.c_int), ("chunk", ctypes.c_int),
                ("cutoff_sigma", ctypes.c_float), ("reduction", ctypes.c_int)]


class GsFFT(ctypes.Structure):
    _fields_ = [("r2c", ctypes.c_int), ("c2r", ctypes.c_int), ("D", ctypes.c_int), ("B", ctypes.c_int),
                ("work_bytes", ctypes.c_size_t), ("r2c_rows", ctypes.c_int), ("c2r_rows", ctypes.c_int)]


class GsFSC(ctypes.Structure):
    _fields_ = [("r2c", ctypes.c_int), ("D", ctypes.c_int), ("work_bytes", ctypes.c_size_t)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgs.so not built ({LIB_PATH}); run python -m paper_2508_04929_b300.build")
    return ctypes.CDLL(LIB_PATH)


lib = _load()

_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_S = ctypes.c_size_t
_CFG = ctypes.POINTER(GsConfig)
_SIGS = {
    "gs_tiles_per_image": [_CFG, ctypes.POINTER(_I)],
    "gs_proj_size": [_I, _I, ctypes.POINTER(_S)],
    "gs_workspace_size": [_CFG, _I, _I, _S, ctypes.POINTER(_S)],
    "gs_fft_create": [_I, _I, ctypes.POINTER(GsFFT)],
    "gs_fft_destroy": [ctypes.POINTER(GsFFT)],
    "gs_read_status": [_P, _P, _I, ctypes.POINTER(_I)],
    "gs_clear_status": [_P, _P],
    "gs_project": [_CFG, _P, _I, _P, _I, _P, _P, _S, _P],
    "gs_bin_sort": [_CFG, _P, _I, _I, _P, _S, _P, _S, _P, _P, _P],
    "gs_render_fwd": [_CFG, _P, _I, _P, _P, _I, _P, _P],
    "gs_apply_ctf": [_CFG, _P, _P, _I, _P, ctypes.POINTER(GsFFT), _P, _S, _P],
    "gs_loss": [_CFG, _P, _P, _I, _P, _P, _P],
    "gs_ctf_loss_grad": [_CFG, _P, _P, _P, _I, _P, _P, ctypes.POINTER(GsFFT), _P, _S, _P],
    "gs_render_bwd": [_CFG, _P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _S, _P],
    "gs_render_bwd_pose": [_CFG, _P, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P, _S, _P],
    "gs_step": [_P, _P, _P, _P, _I, _I, _F, _F, _F, _F, _P],
    "gs_step_counted": [_P, _P, _P, _P, _I, _P, _F, _F, _F, _F, _P],
    "gs_bin_sort_noalloc": [_CFG, _P, _I, _I, _P, _S, _P, _P, _P, ctypes.POINTER(_S)],
    "gs_backproject": [_P, _P, _I, _I, _F, _I, _P, _P],
    "gs_mass_estimate": [_P, _P, _I, _I, _F, _P, _P, _P],
    "gs_seed_sample": [_P, _I, _F, _P, _I, _P, _P, _P, _P, _P],
    "gs_seed_features": [_P, _I, _F, _P, _P, _I, _P, _P],
    "gs_merge_labels": [_P, _I, _P, _I, _I, _F, _P, _P, _P, _P, _P],
    "gs_decode_seeds": [_P, _P, _I, _I, _F, _P, _P, _P],
    "gs_mlp_param_count": [_I, _I, _I, ctypes.POINTER(_S)],
    "gs_mlp_forward": [_P, _I, _I, _I, _P, _P, _I, _P, _P, _P],
    "gs_mlp_backward": [_P, _I, _I, _I, _P, _P, _I, _P, _P, _P, _P, _P],
    "gs_mse": [_P, _P, _P, _I, _I, _F, _P, _P, _P],
    "gs_fourier_shift": [_CFG, _P, _P, _I, _P, ctypes.POINTER(GsFFT), _P, _S, _P],
    "gs_split_gaussians": [_P, _I, _F, _P, _P],
    "gs_voxel_workspace_size": [_I, ctypes.POINTER(_S)],
    "gs_voxelize": [_P, _I, _I, _F, _F, _P, _P, _S, _P],
    "gs_fsc_create": [_I, ctypes.POINTER(GsFSC)],
    "gs_fsc_destroy": [ctypes.POINTER(GsFSC)],
    "gs_fsc_workspace_size": [ctypes.POINTER(GsFSC), ctypes.POINTER(_S)],
    "gs_fsc": [ctypes.POINTER(GsFSC), _P, _P, _P, _P, _S, _P],
}
for _name, _args in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = ctypes.c_int

EXPORTED = tuple(_SIGS)


def _check(name, rc):
    if rc != GS_OK:
        raise GsError(name, rc)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def config(D, E=0.5, tile=16, chunk=128, cutoff_sigma=3.0, reduction=0) -> GsConfig:
    return GsConfig(int(D), float(E), int(tile), int(chunk), float(cutoff_sigma), int(reduction))


def gs_tiles_per_image(cfg: GsConfig) -> int:
    n = _I()
    _check("gs_tiles_per_image", lib.gs_tiles_per_image(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def gs_proj_size(B: int, N: int) -> int:
    """Bytes of gs_project's output buffer: B*N records, the B*N-box plane, the B*N centre low parts."""
    n = _S()
    _check("gs_proj_size", lib.gs_proj_size(B, N, ctypes.byref(n)))
    return n.value


def _check_proj(name, proj, B, N):
    if proj is not None and B > 0 and N > 0 and proj.numel() * proj.element_size() < gs_proj_size(B, N):
        raise ValueError(f"{name}: proj holds {proj.numel() * proj.element_size()} bytes, "
                         f"gs_proj_size({B}, {N}) = {gs_proj_size(B, N)}")


def gs_workspace_size(cfg: GsConfig, B: int, N: int, fft_work_bytes: int = 0) -> int:
    n = _S()
    _check("gs_workspace_size", lib.gs_workspace_size(ctypes.byref(cfg), B, N, fft_work_bytes, ctypes.byref(n)))
    return n.value


def gs_fft_create(D: int, B: int) -> GsFFT:
    f = GsFFT()
    _check("gs_fft_create", lib.gs_fft_create(D, B, ctypes.byref(f)))
    return f


def gs_fft_destroy(f: GsFFT) -> None:
    _check("gs_fft_destroy", lib.gs_fft_destroy(ctypes.byref(f)))


def gs_read_status(ws, clear=True, stream=None) -> int:
    st = _I()
    _check("gs_read_status", lib.gs_read_status(_ptr(ws), _stream(stream), int(clear), ctypes.byref(st)))
    return st.value


def gs_clear_status(ws, stream=None) -> None:
    _check("gs_clear_status", lib.gs_clear_status(_ptr(ws), _stream(stream)))


def gs_project(cfg, theta, W, proj, ws, stream=None) -> None:
    N, B = theta.shape[0], W.shape[0]
    _check_proj("gs_project", proj, B, N)
    _check("gs_project", lib.gs_project(ctypes.byref(cfg), _ptr(theta), N, _ptr(W), B, _ptr(proj), _ptr(ws),
                                        ws.numel() * ws.element_size(), _stream(stream)))


def gs_bin_sort(cfg, proj, B, N, ws, pair_gauss, tile_ranges, n_pairs, stream=None) -> None:
    _check_proj("gs_bin_sort", proj, B, N)
    cap = 0 if pair_gauss is None else pair_gauss.numel()
    _check("gs_bin_sort", lib.gs_bin_sort(ctypes.byref(cfg), _ptr(proj), B, N, _ptr(ws),
                                          ws.numel() * ws.element_size(), _ptr(pair_gauss), cap,
                                          _ptr(tile_ranges), _ptr(n_pairs), _stream(stream)))


def gs_render_fwd(cfg, proj, N, pair_gauss, tile_ranges, B, Q, stream=None) -> None:
    _check("gs_render_fwd", lib.gs_render_fwd(ctypes.byref(cfg), _ptr(proj), N, _ptr(pair_gauss),
                                              _ptr(tile_ranges), B, _ptr(Q), _stream(stream)))


def gs_apply_ctf(cfg, inp, ctf, out, fft, ws, stream=None) -> None:
    B = inp.shape[0]
    _check("gs_apply_ctf", lib.gs_apply_ctf(ctypes.byref(cfg), _ptr(inp), _ptr(ctf), B, _ptr(out),
                                            ctypes.byref(fft), _ptr(ws), ws.numel() * ws.element_size(),
                                            _stream(stream)))


def gs_loss(cfg, X, Y, loss, dLdX=None, stream=None) -> None:
    _check("gs_loss", lib.gs_loss(ctypes.byref(cfg), _ptr(X), _ptr(Y), X.shape[0], _ptr(loss), _ptr(dLdX),
                                  _stream(stream)))


def gs_ctf_loss_grad(cfg, Q, Y, ctf, loss, dLdQ, fft, ws, stream=None) -> None:
    """CTF, loss and adjoint CTF of a training step: loss[B] and dLdQ, without X."""
    _check("gs_ctf_loss_grad", lib.gs_ctf_loss_grad(ctypes.byref(cfg), _ptr(Q), _ptr(Y), _ptr(ctf), Q.shape[0],
                                                    _ptr(loss), _ptr(dLdQ), ctypes.byref(fft), _ptr(ws),
                                                    ws.numel() * ws.element_size(), _stream(stream)))


def gs_render_bwd(cfg, theta, W, proj, pair_gauss, tile_ranges, dLdQ, dtheta, ws, stream=None) -> None:
    N, B = theta.shape[0], W.shape[0]
    _check("gs_render_bwd", lib.gs_render_bwd(ctypes.byref(cfg), _ptr(theta), N, _ptr(W), B, _ptr(proj),
                                              _ptr(pair_gauss), _ptr(tile_ranges), _ptr(dLdQ), _ptr(dtheta),
                                              _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def gs_render_bwd_pose(cfg, theta, W, proj, pair_gauss, tile_ranges, dLdQ, dtheta, dpose, ws, stream=None) -> None:
    """gs_render_bwd plus dL/dW (dpose[:, 0:9]) and dL/dt (dpose[:, 10:12]), accumulated."""
    N, B = theta.shape[0], W.shape[0]
    _check("gs_render_bwd_pose", lib.gs_render_bwd_pose(ctypes.byref(cfg), _ptr(theta), N, _ptr(W), B, _ptr(proj),
                                                        _ptr(pair_gauss), _ptr(tile_ranges), _ptr(dLdQ),
                                                        _ptr(dtheta), _ptr(dpose), _ptr(ws),
                                                        ws.numel() * ws.element_size(), _stream(stream)))


def gs_step(theta, dtheta, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    _check("gs_step", lib.gs_step(_ptr(theta), _ptr(dtheta), _ptr(m), _ptr(v), theta.numel(), int(t), float(lr),
                                  float(beta1), float(beta2), float(eps), _stream(stream)))


def gs_step_counted(theta, dtheta, m, v, t_dev, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    _check("gs_step_counted", lib.gs_step_counted(_ptr(theta), _ptr(dtheta), _ptr(m), _ptr(v), theta.numel(),
                                                  _ptr(t_dev), float(lr), float(beta1), float(beta2), float(eps),
                                                  _stream(stream)))


def gs_bin_sort_noalloc(cfg, proj, B, N, pair_gauss, tile_ranges, n_pairs, stream=None) -> int:
    """Binning and sort with the library's own fixed device scratch (no workspace, no
    allocation).  Returns the scratch bytes this size needs."""
    cap = 0 if pair_gauss is None else pair_gauss.numel()
    need = _S()
    _check("gs_bin_sort_noalloc", lib.gs_bin_sort_noalloc(ctypes.byref(cfg), _ptr(proj), B, N, _ptr(pair_gauss), cap,
                                                          _ptr(tile_ranges), _ptr(n_pairs), _stream(stream),
                                                          ctypes.byref(need)))
    return need.value


# ---------------------------------------------------------------------------------------
# Learned warm start
# ---------------------------------------------------------------------------------------
def gs_backproject(images, W, Dv, vol, E=0.5, stream=None) -> None:
    B, D = images.shape[0], images.shape[-1]
    _check("gs_backproject", lib.gs_backproject(_ptr(images), _ptr(W), B, D, float(E), int(Dv), _ptr(vol),
                                                _stream(stream)))


def gs_mass_estimate(images, ctf, scratch, mass, E=0.5, stream=None) -> None:
    B, D = images.shape[0], images.shape[-1]
    _check("gs_mass_estimate", lib.gs_mass_estimate(_ptr(images), _ptr(ctf), B, D, float(E), _ptr(scratch),
                                                    _ptr(mass), _stream(stream)))


def gs_seed_sample(vol, u, cdf, vmax, pos, voxel=None, E=0.5, stream=None) -> None:
    Dv, K = vol.shape[-1], u.shape[0]
    _check("gs_seed_sample", lib.gs_seed_sample(_ptr(vol), Dv, float(E), _ptr(u), K, _ptr(cdf), _ptr(vmax),
                                                _ptr(voxel), _ptr(pos), _stream(stream)))


def gs_seed_features(vol, vmax, pos, feats, E=0.5, stream=None) -> None:
    Dv, K = vol.shape[-1], pos.shape[0]
    _check("gs_seed_features", lib.gs_seed_features(_ptr(vol), Dv, float(E), _ptr(vmax), _ptr(pos), K,
                                                    _ptr(feats), _stream(stream)))


def gs_merge_labels(pos, theta_fit, Dv, mass, labels, assign=None, moments=None, E=0.5, stream=None) -> None:
    K, N = pos.shape[0], theta_fit.shape[0]
    if assign is None:
        assign = torch.empty(max(N, 1), dtype=torch.int32, device=pos.device)
    if moments is None:
        moments = torch.empty(K * 10, dtype=torch.float64, device=pos.device)
    _check("gs_merge_labels", lib.gs_merge_labels(_ptr(pos), K, _ptr(theta_fit), N, int(Dv), float(E), _ptr(mass),
                                                  _ptr(assign), _ptr(moments), _ptr(labels), _stream(stream)))


def gs_decode_seeds(pos, pred, Dv, mass, theta, E=0.5, stream=None) -> None:
    _check("gs_decode_seeds", lib.gs_decode_seeds(_ptr(pos), _ptr(pred), pos.shape[0], int(Dv), float(E),
                                                  _ptr(mass), _ptr(theta), _stream(stream)))


def gs_mlp_param_count(din, hidden, dout) -> int:
    n = _S()
    _check("gs_mlp_param_count", lib.gs_mlp_param_count(int(din), int(hidden), int(dout), ctypes.byref(n)))
    return n.value


def gs_mlp_forward(params, dims, X, acts, Y, idx=None, stream=None) -> None:
    din, hidden, dout = dims
    n = Y.shape[0]
    _check("gs_mlp_forward", lib.gs_mlp_forward(_ptr(params), din, hidden, dout, _ptr(X), _ptr(idx), n, _ptr(acts),
                                                _ptr(Y), _stream(stream)))


def gs_mlp_backward(params, dims, X, acts, dY, dparams, scratch, idx=None, stream=None) -> None:
    din, hidden, dout = dims
    n = dY.shape[0]
    _check("gs_mlp_backward", lib.gs_mlp_backward(_ptr(params), din, hidden, dout, _ptr(X), _ptr(idx), n,
                                                  _ptr(acts), _ptr(dY), _ptr(dparams), _ptr(scratch),
                                                  _stream(stream)))


def gs_mse(Y, T, loss, dY=None, idx=None, scale=None, stream=None) -> None:
    n, width = Y.shape
    sc = 1.0 / max(n * width, 1) if scale is None else float(scale)
    _check("gs_mse", lib.gs_mse(_ptr(Y), _ptr(T), _ptr(idx), n, width, sc, _ptr(loss), _ptr(dY), _stream(stream)))


# ---------------------------------------------------------------------------------------
# Evaluation: voxelization and FSC
# ---------------------------------------------------------------------------------------
def gs_voxel_workspace_size(N) -> int:
    n = _S()
    _check("gs_voxel_workspace_size", lib.gs_voxel_workspace_size(int(N), ctypes.byref(n)))
    return n.value


def gs_voxelize(theta, Dv, vol, ws, E=0.5, cutoff_sigma=3.0, stream=None) -> None:
    _check("gs_voxelize", lib.gs_voxelize(_ptr(theta), theta.shape[0], int(Dv), float(E), float(cutoff_sigma),
                                          _ptr(vol), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def gs_fsc_create(D) -> GsFSC:
    f = GsFSC()
    _check("gs_fsc_create", lib.gs_fsc_create(int(D), ctypes.byref(f)))
    return f


def gs_fsc_destroy(f: GsFSC) -> None:
    _check("gs_fsc_destroy", lib.gs_fsc_destroy(ctypes.byref(f)))


def gs_fsc_workspace_size(f: GsFSC) -> int:
    n = _S()
    _check("gs_fsc_workspace_size", lib.gs_fsc_workspace_size(ctypes.byref(f), ctypes.byref(n)))
    return n.value


def gs_fsc(f: GsFSC, vol1, vol2, out, ws, stream=None) -> None:
    _check("gs_fsc", lib.gs_fsc(ctypes.byref(f), _ptr(vol1), _ptr(vol2), _ptr(out), _ptr(ws),
                                ws.numel() * ws.element_size(), _stream(stream)))


# ---------------------------------------------------------------------------------------
# Algorithm 1: FourierShift and SplitGaussian
# ---------------------------------------------------------------------------------------
def gs_fourier_shift(cfg, inp, t, out, fft, ws, stream=None) -> None:
    B = inp.shape[0]
    _check("gs_fourier_shift", lib.gs_fourier_shift(ctypes.byref(cfg), _ptr(inp), _ptr(t), B, _ptr(out),
                                                    ctypes.byref(fft), _ptr(ws), ws.numel() * ws.element_size(),
                                                    _stream(stream)))


def gs_split_gaussians(theta, out, alpha=0.5, stream=None) -> None:
    _check("gs_split_gaussians", lib.gs_split_gaussians(_ptr(theta), theta.shape[0], float(alpha), _ptr(out),
                                                        _stream(stream)))
