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

GS_OK, GS_EINVAL, GS_ENOSPC, GS_ECUDA, GS_ECAPTURE = 0, 1, 2, 3, 4
GS_STATUS_NONFINITE, GS_STATUS_OVERFLOW = 1, 2
RECORD_BYTES = 32

_ERR = {GS_EINVAL: "invalid argument", GS_ENOSPC: "buffer too small", GS_ECUDA: "CUDA/cuFFT failure",
        GS_ECAPTURE: "first call on this device made during stream capture"}


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
    "gs_probe_ex2": [_I, _I, _P, _P, ctypes.POINTER(ctypes.c_double)],
}
for _name, _args in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = ctypes.c_int

EXPORTED = tuple(_SIGS)


def _check(name, rc):
    if rc != GS_OK:
        raise GsError(name, rc)


# dtypes a device argument may have: FP32 arrays, 32-bit integer arrays (pair lists, tile
# ranges, counts, indices), FP64 scratch, and raw byte buffers (workspace, projection) of any dtype
_F32 = (torch.float32,)
_I32 = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())
_F64 = (torch.float64,)
_I64 = (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())
_RAW = None


def _ptr(t, name="", arg="", dtypes=_F32, optional=True):
    """Device pointer of tensor t after checking that the kernels can read it as declared:
    a contiguous CUDA tensor of one of ``dtypes`` (any dtype when None).  None passes a null
    pointer where the C entry point allows one.  Raises ValueError otherwise: a host tensor,
    a strided view or a float64 array would be misread by the kernels, not reported."""
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name}: {arg} is required")
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: {arg} must be a torch tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise ValueError(f"{name}: {arg} must be in CUDA device memory, got device {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: {arg} must be contiguous (got strides {tuple(t.stride())})")
    if dtypes is not None and t.dtype not in dtypes:
        raise ValueError(f"{name}: {arg} must have dtype {' or '.join(str(d) for d in dtypes)}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _rows(t, name, arg, width):
    """Check that t holds rows of ``width`` values (e.g. theta [N, 11], W [B, 9] or [B, 3, 3])."""
    if isinstance(t, torch.Tensor) and (t.dim() == 0 or t.numel() % width != 0 or
                                        (t.dim() >= 2 and t.shape[0] * width != t.numel())):
        raise ValueError(f"{name}: {arg} must hold rows of {width} values, got shape {tuple(t.shape)}")


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
    _check("gs_read_status", lib.gs_read_status(_ptr(ws, "gs_read_status", "ws", _RAW, False), _stream(stream),
                                                int(clear), ctypes.byref(st)))
    return st.value


def gs_clear_status(ws, stream=None) -> None:
    _check("gs_clear_status", lib.gs_clear_status(_ptr(ws, "gs_clear_status", "ws", _RAW, False), _stream(stream)))


def _check_proj(name, proj, B, N):
    if proj is not None and B > 0 and N > 0 and proj.numel() * proj.element_size() < gs_proj_size(B, N):
        raise ValueError(f"{name}: proj holds {proj.numel() * proj.element_size()} bytes, "
                         f"gs_proj_size({B}, {N}) = {gs_proj_size(B, N)}")


def _bytes(t):
    return 0 if t is None else t.numel() * t.element_size()


def gs_project(cfg, theta, W, proj, ws, stream=None) -> None:
    n = "gs_project"
    _rows(theta, n, "theta", 11)
    _rows(W, n, "W", 9)
    N, B = theta.shape[0], W.numel() // 9
    _check_proj(n, proj, B, N)
    _check(n, lib.gs_project(ctypes.byref(cfg), _ptr(theta, n, "theta"), N, _ptr(W, n, "W"), B,
                             _ptr(proj, n, "proj", _RAW), _ptr(ws, n, "ws", _RAW), _bytes(ws), _stream(stream)))


def gs_bin_sort(cfg, proj, B, N, ws, pair_gauss, tile_ranges, n_pairs, stream=None) -> None:
    n = "gs_bin_sort"
    _check_proj(n, proj, B, N)
    cap = 0 if pair_gauss is None else pair_gauss.numel()
    _check(n, lib.gs_bin_sort(ctypes.byref(cfg), _ptr(proj, n, "proj", _RAW), B, N, _ptr(ws, n, "ws", _RAW),
                              _bytes(ws), _ptr(pair_gauss, n, "pair_gauss", _I32), cap,
                              _ptr(tile_ranges, n, "tile_ranges", _I32), _ptr(n_pairs, n, "n_pairs", _I32),
                              _stream(stream)))


def gs_render_fwd(cfg, proj, N, pair_gauss, tile_ranges, B, Q, stream=None) -> None:
    n = "gs_render_fwd"
    _check_proj(n, proj, B, N)
    _check(n, lib.gs_render_fwd(ctypes.byref(cfg), _ptr(proj, n, "proj", _RAW), N,
                                _ptr(pair_gauss, n, "pair_gauss", _I32), _ptr(tile_ranges, n, "tile_ranges", _I32),
                                B, _ptr(Q, n, "Q"), _stream(stream)))


def gs_apply_ctf(cfg, inp, ctf, out, fft, ws, stream=None) -> None:
    n = "gs_apply_ctf"
    _rows(ctf, n, "ctf", 5)
    B = inp.shape[0]
    _check(n, lib.gs_apply_ctf(ctypes.byref(cfg), _ptr(inp, n, "in"), _ptr(ctf, n, "ctf"), B, _ptr(out, n, "out"),
                               ctypes.byref(fft), _ptr(ws, n, "ws", _RAW), _bytes(ws), _stream(stream)))


def gs_loss(cfg, X, Y, loss, dLdX=None, stream=None) -> None:
    n = "gs_loss"
    _check(n, lib.gs_loss(ctypes.byref(cfg), _ptr(X, n, "X"), _ptr(Y, n, "Y"), X.shape[0], _ptr(loss, n, "loss"),
                          _ptr(dLdX, n, "dLdX"), _stream(stream)))


def gs_ctf_loss_grad(cfg, Q, Y, ctf, loss, dLdQ, fft, ws, stream=None) -> None:
    """CTF, loss and adjoint CTF of a training step: loss[B] and dLdQ, without X."""
    n = "gs_ctf_loss_grad"
    _rows(ctf, n, "ctf", 5)
    _check(n, lib.gs_ctf_loss_grad(ctypes.byref(cfg), _ptr(Q, n, "Q"), _ptr(Y, n, "Y"), _ptr(ctf, n, "ctf"),
                                   Q.shape[0], _ptr(loss, n, "loss"), _ptr(dLdQ, n, "dLdQ"), ctypes.byref(fft),
                                   _ptr(ws, n, "ws", _RAW), _bytes(ws), _stream(stream)))


def gs_render_bwd(cfg, theta, W, proj, pair_gauss, tile_ranges, dLdQ, dtheta, ws, stream=None) -> None:
    n = "gs_render_bwd"
    _rows(theta, n, "theta", 11)
    _rows(W, n, "W", 9)
    N, B = theta.shape[0], W.numel() // 9
    _check_proj(n, proj, B, N)
    _check(n, lib.gs_render_bwd(ctypes.byref(cfg), _ptr(theta, n, "theta"), N, _ptr(W, n, "W"), B,
                                _ptr(proj, n, "proj", _RAW), _ptr(pair_gauss, n, "pair_gauss", _I32),
                                _ptr(tile_ranges, n, "tile_ranges", _I32), _ptr(dLdQ, n, "dLdQ"),
                                _ptr(dtheta, n, "dtheta"), _ptr(ws, n, "ws", _RAW), _bytes(ws), _stream(stream)))


def gs_render_bwd_pose(cfg, theta, W, proj, pair_gauss, tile_ranges, dLdQ, dtheta, dpose, ws, stream=None) -> None:
    """gs_render_bwd plus dL/dW (dpose[:, 0:9]) and dL/dt (dpose[:, 10:12]), accumulated."""
    n = "gs_render_bwd_pose"
    _rows(theta, n, "theta", 11)
    _rows(W, n, "W", 9)
    N, B = theta.shape[0], W.numel() // 9
    _check_proj(n, proj, B, N)
    _check(n, lib.gs_render_bwd_pose(ctypes.byref(cfg), _ptr(theta, n, "theta"), N, _ptr(W, n, "W"), B,
                                     _ptr(proj, n, "proj", _RAW), _ptr(pair_gauss, n, "pair_gauss", _I32),
                                     _ptr(tile_ranges, n, "tile_ranges", _I32), _ptr(dLdQ, n, "dLdQ"),
                                     _ptr(dtheta, n, "dtheta"), _ptr(dpose, n, "dpose"), _ptr(ws, n, "ws", _RAW),
                                     _bytes(ws), _stream(stream)))


def gs_step(theta, dtheta, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    n = "gs_step"
    _check(n, lib.gs_step(_ptr(theta, n, "theta"), _ptr(dtheta, n, "dtheta"), _ptr(m, n, "m"), _ptr(v, n, "v"),
                          theta.numel(), int(t), float(lr), float(beta1), float(beta2), float(eps), _stream(stream)))


def gs_step_counted(theta, dtheta, m, v, t_dev, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    n = "gs_step_counted"
    _check(n, lib.gs_step_counted(_ptr(theta, n, "theta"), _ptr(dtheta, n, "dtheta"), _ptr(m, n, "m"),
                                  _ptr(v, n, "v"), theta.numel(), _ptr(t_dev, n, "t_dev", _I32), float(lr),
                                  float(beta1), float(beta2), float(eps), _stream(stream)))


def gs_bin_sort_noalloc(cfg, proj, B, N, pair_gauss, tile_ranges, n_pairs, stream=None) -> int:
    """Binning and sort with the library's own fixed device scratch (no workspace, no
    allocation).  Returns the scratch bytes this size needs."""
    n = "gs_bin_sort_noalloc"
    cap = 0 if pair_gauss is None else pair_gauss.numel()
    need = _S()
    _check(n, lib.gs_bin_sort_noalloc(ctypes.byref(cfg), _ptr(proj, n, "proj", _RAW), B, N,
                                      _ptr(pair_gauss, n, "pair_gauss", _I32), cap,
                                      _ptr(tile_ranges, n, "tile_ranges", _I32), _ptr(n_pairs, n, "n_pairs", _I32),
                                      _stream(stream), ctypes.byref(need)))
    return need.value


# ---------------------------------------------------------------------------------------
# Learned warm start
# ---------------------------------------------------------------------------------------
def gs_backproject(images, W, Dv, vol, E=0.5, stream=None) -> None:
    B, D = images.shape[0], images.shape[-1]
    n = "gs_backproject"
    _check(n, lib.gs_backproject(_ptr(images, n, "images"), _ptr(W, n, "W"), B, D, float(E), int(Dv),
                                 _ptr(vol, n, "vol"), _stream(stream)))


def gs_mass_estimate(images, ctf, scratch, mass, E=0.5, stream=None) -> None:
    B, D = images.shape[0], images.shape[-1]
    n = "gs_mass_estimate"
    _check(n, lib.gs_mass_estimate(_ptr(images, n, "images"), _ptr(ctf, n, "ctf"), B, D, float(E),
                                   _ptr(scratch, n, "scratch", _F64), _ptr(mass, n, "mass"), _stream(stream)))


def gs_seed_sample(vol, u, cdf, vmax, pos, voxel=None, E=0.5, stream=None) -> None:
    Dv, K = vol.shape[-1], u.shape[0]
    n = "gs_seed_sample"
    _check(n, lib.gs_seed_sample(_ptr(vol, n, "vol"), Dv, float(E), _ptr(u, n, "u"), K, _ptr(cdf, n, "cdf", _I64),
                                 _ptr(vmax, n, "vmax"), _ptr(voxel, n, "voxel", _I32), _ptr(pos, n, "pos"),
                                 _stream(stream)))


def gs_seed_features(vol, vmax, pos, feats, E=0.5, stream=None) -> None:
    Dv, K = vol.shape[-1], pos.shape[0]
    n = "gs_seed_features"
    _check(n, lib.gs_seed_features(_ptr(vol, n, "vol"), Dv, float(E), _ptr(vmax, n, "vmax"), _ptr(pos, n, "pos"), K,
                                   _ptr(feats, n, "feats"), _stream(stream)))


def gs_merge_labels(pos, theta_fit, Dv, mass, labels, assign=None, moments=None, E=0.5, stream=None) -> None:
    K, N = pos.shape[0], theta_fit.shape[0]
    if assign is None:
        assign = torch.empty(max(N, 1), dtype=torch.int32, device=pos.device)
    if moments is None:
        moments = torch.empty(K * 10, dtype=torch.float64, device=pos.device)
    n = "gs_merge_labels"
    _check(n, lib.gs_merge_labels(_ptr(pos, n, "pos"), K, _ptr(theta_fit, n, "theta_fit"), N, int(Dv), float(E),
                                  _ptr(mass, n, "mass"), _ptr(assign, n, "assign", _I32),
                                  _ptr(moments, n, "moments", _F64), _ptr(labels, n, "labels"), _stream(stream)))


def gs_decode_seeds(pos, pred, Dv, mass, theta, E=0.5, stream=None) -> None:
    n = "gs_decode_seeds"
    _check(n, lib.gs_decode_seeds(_ptr(pos, n, "pos"), _ptr(pred, n, "pred"), pos.shape[0], int(Dv), float(E),
                                  _ptr(mass, n, "mass"), _ptr(theta, n, "theta"), _stream(stream)))


def gs_mlp_param_count(din, hidden, dout) -> int:
    n = _S()
    _check("gs_mlp_param_count", lib.gs_mlp_param_count(int(din), int(hidden), int(dout), ctypes.byref(n)))
    return n.value


def gs_mlp_forward(params, dims, X, acts, Y, idx=None, stream=None) -> None:
    din, hidden, dout = dims
    n = Y.shape[0]
    f = "gs_mlp_forward"
    _check(f, lib.gs_mlp_forward(_ptr(params, f, "params"), din, hidden, dout, _ptr(X, f, "X"),
                                 _ptr(idx, f, "idx", _I32), n, _ptr(acts, f, "acts"), _ptr(Y, f, "Y"),
                                 _stream(stream)))


def gs_mlp_backward(params, dims, X, acts, dY, dparams, scratch, idx=None, stream=None) -> None:
    din, hidden, dout = dims
    n = dY.shape[0]
    f = "gs_mlp_backward"
    _check(f, lib.gs_mlp_backward(_ptr(params, f, "params"), din, hidden, dout, _ptr(X, f, "X"),
                                  _ptr(idx, f, "idx", _I32), n, _ptr(acts, f, "acts"), _ptr(dY, f, "dY"),
                                  _ptr(dparams, f, "dparams"), _ptr(scratch, f, "scratch"), _stream(stream)))


def gs_mse(Y, T, loss, dY=None, idx=None, scale=None, stream=None) -> None:
    n, width = Y.shape
    sc = 1.0 / max(n * width, 1) if scale is None else float(scale)
    f = "gs_mse"
    _check(f, lib.gs_mse(_ptr(Y, f, "Y"), _ptr(T, f, "T"), _ptr(idx, f, "idx", _I32), n, width, sc,
                         _ptr(loss, f, "loss"), _ptr(dY, f, "dY"), _stream(stream)))


# ---------------------------------------------------------------------------------------
# Evaluation: voxelization and FSC
# ---------------------------------------------------------------------------------------
def gs_voxel_workspace_size(N) -> int:
    n = _S()
    _check("gs_voxel_workspace_size", lib.gs_voxel_workspace_size(int(N), ctypes.byref(n)))
    return n.value


def gs_voxelize(theta, Dv, vol, ws, E=0.5, cutoff_sigma=3.0, stream=None) -> None:
    n = "gs_voxelize"
    _rows(theta, n, "theta", 11)
    _check(n, lib.gs_voxelize(_ptr(theta, n, "theta"), theta.shape[0], int(Dv), float(E), float(cutoff_sigma),
                              _ptr(vol, n, "vol"), _ptr(ws, n, "ws", _RAW), _bytes(ws), _stream(stream)))


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
    n = "gs_fsc"
    _check(n, lib.gs_fsc(ctypes.byref(f), _ptr(vol1, n, "vol1"), _ptr(vol2, n, "vol2"), _ptr(out, n, "out"),
                         _ptr(ws, n, "ws", _RAW), _bytes(ws), _stream(stream)))


# ---------------------------------------------------------------------------------------
# Algorithm 1: FourierShift and SplitGaussian
# ---------------------------------------------------------------------------------------
def gs_fourier_shift(cfg, inp, t, out, fft, ws, stream=None) -> None:
    B = inp.shape[0]
    n = "gs_fourier_shift"
    _check(n, lib.gs_fourier_shift(ctypes.byref(cfg), _ptr(inp, n, "in"), _ptr(t, n, "t"), B, _ptr(out, n, "out"),
                                   ctypes.byref(fft), _ptr(ws, n, "ws", _RAW), _bytes(ws), _stream(stream)))


def gs_split_gaussians(theta, out, alpha=0.5, stream=None) -> None:
    n = "gs_split_gaussians"
    _rows(theta, n, "theta", 11)
    _check(n, lib.gs_split_gaussians(_ptr(theta, n, "theta"), theta.shape[0], float(alpha), _ptr(out, n, "out"),
                                     _stream(stream)))


# ---------------------------------------------------------------------------------------
# Diagnostics
# ---------------------------------------------------------------------------------------
def gs_probe_ex2(blocks, iters, sink, stream=None) -> float:
    """Launch the ex2.approx throughput probe; returns the number of ex2 it executes (the
    caller times the launch)."""
    n = "gs_probe_ex2"
    cnt = ctypes.c_double()
    _check(n, lib.gs_probe_ex2(int(blocks), int(iters), _ptr(sink, n, "sink", optional=False), _stream(stream),
                               ctypes.byref(cnt)))
    return cnt.value

