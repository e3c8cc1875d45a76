"""Python binding of libgbmg.so (C ABI in include/gbmg.h).

Argument marshalling only: every step of the multigrid hot path runs in the
library's CUDA kernels.  Functions carry the C names; tensors are PyTorch
CUDA tensors (complex128 / complex64) whose data pointers are passed
through, and the stream defaults to torch's current stream.  Importing
this module loads the shared library and raises if it has not been built
(``python paper_1612_07873_gb300/build.py``): there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

MG_MAX_LEVELS = 4
F64, F32, BF16, F16, I16 = 0, 1, 2, 3, 4
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "out of device memory",
          -4: "call out of order", -5: "solver did not converge", -6: "numerical breakdown",
          -7: "device wait timed out", -8: "rank-deficient null-vector block"}
MG_ERR_ARG = -1
MG_ERR_CUDA = -2
MG_ERR_OOM = -3
MG_ERR_STATE = -4
MG_ERR_NOT_CONVERGED = -5
MG_ERR_NUMERICAL = -6
MG_ERR_TIMEOUT = -7
MG_ERR_RANK = -8


class mg_params(C.Structure):
    _fields_ = [
        ("dims", C.c_int * 4),
        ("t_antiperiodic", C.c_int),
        ("mass", C.c_double),
        ("csw", C.c_double),
        ("nlevels", C.c_int),
        ("block", (C.c_int * 4) * MG_MAX_LEVELS),
        ("nvec", C.c_int * MG_MAX_LEVELS),
        ("setup_sweeps", C.c_int),
        ("seed", C.c_uint64),
        ("prec_fine", C.c_int),
        ("prec_coarse", C.c_int),
        ("mr_iters", C.c_int),
        ("mr_omega", C.c_double),
        ("gcr_nkrylov", C.c_int),
        ("inner_tol", C.c_double),
        ("inner_maxiter", C.c_int),
        ("coarse_tol", C.c_double),
        ("coarse_maxiter", C.c_int),
        ("link_slots", C.c_int),
        ("red_black", C.c_int),
        ("prec_smoother", C.c_int),
    ]


class mg_solve_stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("restarts", C.c_int),
        ("level_iters", C.c_int * MG_MAX_LEVELS),
        ("true_residual", C.c_double),
        ("seconds", C.c_double),
        ("history_len", C.c_int),
        ("history", C.c_double * 512),
    ]


def _load():
    path = _build.lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libgbmg.so not built ({path}); run "
                          "`python paper_1612_07873_gb300/build.py`")
    lib = C.CDLL(path)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    sig = {
        "mg_default_params": (None, [C.POINTER(mg_params)]),
        "mg_create": (i, [C.POINTER(mg_params), vp, C.POINTER(vp)]),
        "mg_destroy": (i, [vp]),
        "mg_setup_nullvecs": (i, [vp, i, vp, vp]),
        "mg_set_nullvecs": (i, [vp, i, vp, vp]),
        "mg_get_nullvecs": (i, [vp, i, i, vp, sz, vp]),
        "mg_build_coarse": (i, [vp, i, vp]),
        "mg_coarse_apply": (i, [vp, i, vp, vp, i, vp]),
        "mg_apply": (i, [vp, i, vp, vp, vp]),
        "mg_wilson_clover_apply": (i, [vp, vp, vp, vp]),
        "mg_restrict": (i, [vp, i, vp, vp, vp]),
        "mg_prolong": (i, [vp, i, vp, vp, vp]),
        "mg_gcr_solve": (i, [vp, vp, vp, d, i, C.POINTER(mg_solve_stats), vp]),
        "mg_gcr_solve_multi": (i, [vp, vp, vp, i, d, i, C.POINTER(mg_solve_stats), vp]),
        "mg_tune_set": (i, [C.c_char_p, i]),
        "mg_save": (i, [vp, C.c_char_p]),
        "mg_load": (i, [vp, C.c_char_p]),
        "mg_inject_fault": (i, [vp, C.c_char_p, i]),
        "mg_inner_product": (i, [vp, i, vp, vp, i, i, C.POINTER(C.c_double), vp]),
        "mg_wilson_clover_apply_multi": (i, [vp, vp, vp, i, vp]),
        "mg_wilson_clover_apply_bf16": (i, [vp, vp, vp, i, vp]),
        "mg_schur_apply": (i, [vp, i, vp, vp, i, vp]),
        "mg_tune_get": (i, [C.c_char_p]),
        "mg_tune_report": (i, [C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_float), i]),
        "mg_get_coarse_links": (i, [vp, i, vp, sz, vp]),
        "mg_set_coarse_links": (i, [vp, i, vp, sz, vp]),
        "mg_level_info": (i, [vp, i, C.POINTER(C.c_int), C.POINTER(C.c_int),
                              C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "mg_gauge_compression": (i, [vp, C.POINTER(C.c_int), C.POINTER(d), C.POINTER(d)]),
        "mg_profile_enable": (i, [vp, i]),
        "mg_profile_reset": (i, [vp]),
        "mg_profile_query": (i, [vp, C.c_char_p, i, C.POINTER(C.c_int), C.POINTER(d),
                                 C.POINTER(d), C.POINTER(d)]),
        "mg_block_orthonormalise_noalloc": (i, [vp, vp, sz, C.POINTER(C.c_int),
                                                C.POINTER(C.c_int), i, i, vp]),
        "mg_device_status": (i, [vp, vp]),
        "mg_set_setup_sweeps": (i, [vp, i]),
        "mg_coarse_apply_multi": (i, [C.POINTER(vp), C.POINTER(C.c_int), C.POINTER(vp),
                                      C.POINTER(vp), i, i, vp]),
        "mg_cnn_create": (i, [i, C.c_uint64, C.POINTER(vp)]),
        "mg_cnn_destroy": (i, [vp]),
        "mg_cnn_nparams": (i, [vp, C.POINTER(C.c_int)]),
        "mg_cnn_get_params": (i, [vp, vp, sz, i, vp]),
        "mg_cnn_set_params": (i, [vp, vp, sz, vp]),
        "mg_cnn_forward": (i, [vp, C.POINTER(C.c_int), vp, vp, vp]),
        "mg_cnn_loss_grad": (i, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), vp, vp,
                                 C.POINTER(d), vp]),
        "mg_cnn_adam_step": (i, [vp, C.c_float, vp]),
        "mg_launch_count": (C.c_longlong, [vp]),
        "mg_fma_peak": (i, [i, C.POINTER(d), vp]),
        "mg_halo_plan": (i, [C.POINTER(C.c_int), C.POINTER(C.c_int), i, C.POINTER(C.c_int),
                             C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "mg_halo_face_sites": (i, [C.POINTER(C.c_int), i, i, C.POINTER(C.c_int)]),
        "mg_halo_create": (i, [vp, i, C.POINTER(C.c_int), C.POINTER(vp), vp]),
        "mg_halo_destroy": (i, [vp]),
        "mg_halo_info": (i, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                             C.POINTER(sz)]),
        "mg_halo_scatter": (i, [vp, i, vp, vp, i, vp]),
        "mg_halo_pack": (i, [vp, i, vp, vp]),
        "mg_halo_exchange": (i, [vp, vp]),
        "mg_halo_apply": (i, [vp, i, vp, vp, vp]),
        "mg_halo_buffers": (i, [vp, i, C.POINTER(vp), C.POINTER(vp)]),
        "mg_halo_launch_count": (C.c_longlong, [vp]),
        "mg_status_string": (C.c_char_p, [i]),
        "mg_last_error": (C.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()
LIB_PATH = _build.lib_path()


class MGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ok(st, ctx=None):
    if st != 0:
        msg = LIB.mg_last_error(ctx)
        raise MGError(st, msg.decode() if msg else "")


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expects a contiguous CUDA tensor"
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def default_params(**kw) -> mg_params:
    p = mg_params()
    LIB.mg_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "dims":
            p.dims[:] = list(v)
        elif k == "block":
            for l, b in enumerate(v):
                p.block[l][:] = list(b)
        elif k == "nvec":
            for l, n in enumerate(v):
                p.nvec[l] = n
        else:
            setattr(p, k, v)
    return p


def mg_create(params: mg_params, gauge: torch.Tensor):
    assert gauge.dtype == torch.complex128
    h = C.c_void_p()
    _ok(LIB.mg_create(C.byref(params), _ptr(gauge), C.byref(h)))
    return h


def mg_destroy(ctx):
    _ok(LIB.mg_destroy(ctx))


def mg_setup_nullvecs(ctx, level, init=None, stream=None):
    _ok(LIB.mg_setup_nullvecs(ctx, level, _ptr(init), _stream(stream)), ctx)


def mg_set_nullvecs(ctx, level, vecs, stream=None):
    assert vecs.dtype == torch.complex128
    _ok(LIB.mg_set_nullvecs(ctx, level, _ptr(vecs), _stream(stream)), ctx)


def mg_get_nullvecs(ctx, level, out, kind=1, stream=None):
    _ok(LIB.mg_get_nullvecs(ctx, level, kind, _ptr(out), out.numel() * out.element_size(),
                            _stream(stream)), ctx)
    return out


def mg_build_coarse(ctx, level, stream=None):
    _ok(LIB.mg_build_coarse(ctx, level, _stream(stream)), ctx)


def mg_coarse_apply(ctx, level, y, x, nrhs=1, stream=None):
    _ok(LIB.mg_coarse_apply(ctx, level, _ptr(y), _ptr(x), nrhs, _stream(stream)), ctx)


def mg_apply(ctx, level, y, x, stream=None):
    _ok(LIB.mg_apply(ctx, level, _ptr(y), _ptr(x), _stream(stream)), ctx)


def mg_wilson_clover_apply(ctx, out, inp, stream=None):
    _ok(LIB.mg_wilson_clover_apply(ctx, _ptr(out), _ptr(inp), _stream(stream)), ctx)


def mg_wilson_clover_apply_multi(ctx, out, inp, nrhs, stream=None):
    """out[v] = M inp[v] for nrhs fine vectors stored back to back."""
    _ok(LIB.mg_wilson_clover_apply_multi(ctx, _ptr(out), _ptr(inp), nrhs, _stream(stream)), ctx)


def mg_wilson_clover_apply_bf16(ctx, out, inp, nrhs=1, stream=None):
    """The 16-bit smoother's operator; out, inp: bfloat16 tensors [nrhs][V][12][2]."""
    _ok(LIB.mg_wilson_clover_apply_bf16(ctx, _ptr(out), _ptr(inp), nrhs, _stream(stream)), ctx)


def mg_restrict(ctx, level, coarse, fine, stream=None):
    _ok(LIB.mg_restrict(ctx, level, _ptr(coarse), _ptr(fine), _stream(stream)), ctx)


def mg_prolong(ctx, level, fine, coarse, stream=None):
    _ok(LIB.mg_prolong(ctx, level, _ptr(fine), _ptr(coarse), _stream(stream)), ctx)


def mg_gcr_solve(ctx, x, b, tol=1e-10, maxiter=200, stream=None, check=True):
    s = mg_solve_stats()
    st = LIB.mg_gcr_solve(ctx, _ptr(x), _ptr(b), tol, maxiter, C.byref(s), _stream(stream))
    if check:
        _ok(st, ctx)
    return dict(status=st, iters=s.iters, restarts=s.restarts,
                level_iters=list(s.level_iters), true_residual=s.true_residual,
                seconds=s.seconds, history=list(s.history[:s.history_len]))


def mg_gcr_solve_multi(ctx, x, b, nrhs, tol=1e-10, maxiter=200, stream=None, check=True):
    """x, b: [nrhs][V][12] complex128 on the device.  Returns one stats dict
    per right-hand side."""
    recs = (mg_solve_stats * nrhs)()
    st = LIB.mg_gcr_solve_multi(ctx, _ptr(x), _ptr(b), nrhs, tol, maxiter, recs,
                                _stream(stream))
    if check:
        _ok(st, ctx)
    return [dict(status=st, iters=s.iters, restarts=s.restarts,
                 level_iters=list(s.level_iters), true_residual=s.true_residual,
                 seconds=s.seconds, history=list(s.history[:s.history_len])) for s in recs]


def mg_schur_apply(ctx, level, y, x, nrhs=1, stream=None):
    """y_o = S x_o on compact odd-parity vectors [nrhs][V/2][ndof]."""
    _ok(LIB.mg_schur_apply(ctx, level, _ptr(y), _ptr(x), nrhs, _stream(stream)), ctx)


def mg_save(ctx, path):
    """Write the setup (null vectors, coarse links) of every level to path."""
    _ok(LIB.mg_save(ctx, str(path).encode()), ctx)


def mg_load(ctx, path):
    """Restore a setup written by mg_save into a matching context."""
    _ok(LIB.mg_load(ctx, str(path).encode()), ctx)


def mg_tune_set(key, choice):
    """Pin the autotuner's choice for `key` (choice < 0: forget it)."""
    _ok(LIB.mg_tune_set(key.encode(), int(choice)), None)


def mg_tune_get(key):
    return LIB.mg_tune_get(key.encode())


def mg_tune_report(key):
    """[(choice, ms per launch)] of the last tuning of `key` in this process."""
    n = LIB.mg_tune_report(key.encode(), None, None, 0)
    if n <= 0:
        return []
    ch, ms = (C.c_int * n)(), (C.c_float * n)()
    LIB.mg_tune_report(key.encode(), ch, ms, n)
    return list(zip(list(ch), [float(v) for v in ms]))


def mg_get_coarse_links(ctx, level, out, stream=None):
    _ok(LIB.mg_get_coarse_links(ctx, level, _ptr(out), out.numel() * out.element_size(),
                                _stream(stream)), ctx)
    return out


def mg_set_coarse_links(ctx, level, links, stream=None):
    assert links.dtype == torch.complex128
    _ok(LIB.mg_set_coarse_links(ctx, level, _ptr(links), links.numel() * links.element_size(),
                                _stream(stream)), ctx)


def mg_level_info(ctx, level):
    dims = (C.c_int * 4)()
    vol, nd, vp = C.c_int(), C.c_int(), C.c_int()
    _ok(LIB.mg_level_info(ctx, level, dims, C.byref(vol), C.byref(nd), C.byref(vp)), ctx)
    return dict(dims=tuple(dims), volume=vol.value, ndof=nd.value,
                dtype=torch.complex128 if vp.value == F64 else torch.complex64)


def mg_gauge_compression(ctx):
    """Eligible compressed link forms of the FP32 fine operator and the
    8-real form's reconstruction error (largest, root-mean-square)."""
    f, mx, rms = C.c_int(), C.c_double(), C.c_double()
    _ok(LIB.mg_gauge_compression(ctx, C.byref(f), C.byref(mx), C.byref(rms)), ctx)
    return dict(two_row=bool(f.value & 1), eight_real=bool(f.value & 2), max_dev8=mx.value,
                rms_dev8=rms.value)


def mg_profile_enable(ctx, on=True):
    _ok(LIB.mg_profile_enable(ctx, int(on)), ctx)


def mg_profile_reset(ctx):
    _ok(LIB.mg_profile_reset(ctx), ctx)


def mg_profile_query(ctx, name, level=-1):
    n, ms, b, f = C.c_int(), C.c_double(), C.c_double(), C.c_double()
    _ok(LIB.mg_profile_query(ctx, name.encode(), level, C.byref(n), C.byref(ms), C.byref(b),
                             C.byref(f)), ctx)
    return dict(launches=n.value, ms=ms.value, bytes=b.value, flops=f.value)


def mg_block_orthonormalise_noalloc(vecs, out, dims, block, stream=None):
    """Context-free block orthonormalisation that allocates no device memory
    (for callers that cannot let the library allocate); vecs, out:
    [nvec][V][ndof] complex128 CUDA tensors of the same shape on the current
    device."""
    assert vecs.dtype == torch.complex128 and out.dtype == torch.complex128
    assert vecs.dim() == 3 and out.shape == vecs.shape, "out must have the shape of vecs"
    dev = torch.cuda.current_device()
    assert vecs.device == out.device and vecs.device.index == dev, \
        "vecs and out must be on the current CUDA device"
    nvec, vol, ndof = vecs.shape
    d = (C.c_int * 4)(*dims)
    b = (C.c_int * 4)(*block)
    st = LIB.mg_block_orthonormalise_noalloc(_ptr(vecs), _ptr(out),
                                             out.numel() * out.element_size(), d, b, ndof, nvec,
                                             _stream(stream))
    _ok(st, None)
    return out


def mg_device_status(ctx, stream=None):
    _ok(LIB.mg_device_status(ctx, _stream(stream)), ctx)


def mg_inner_product(ctx, level, a, b, fp64=True, stream=None):
    """sum conj(a) b over one level vector (complex64 or complex128 tensors)
    with the solvers' accumulation; returns a Python complex."""
    prec = {torch.complex64: 1, torch.complex128: 0}[a.dtype]
    assert b.dtype == a.dtype and a.is_contiguous() and b.is_contiguous()
    out = (C.c_double * 2)()
    _ok(LIB.mg_inner_product(ctx, level, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                             prec, int(bool(fp64)), out, _stream(stream)), ctx)
    return complex(out[0], out[1])


def mg_inject_fault(ctx, what, count=1):
    """Host-side fault injection for error-path tests ("coarse_mma_wait")."""
    _ok(LIB.mg_inject_fault(ctx, what.encode(), count), ctx)


def mg_coarse_apply_multi(ctxs, levels, ys, xs, nrhs, stream=None):
    k = len(ctxs)
    c_ctx = (C.c_void_p * k)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    c_lev = (C.c_int * k)(*levels)
    c_y = (C.c_void_p * k)(*[t.data_ptr() for t in ys])
    c_x = (C.c_void_p * k)(*[t.data_ptr() for t in xs])
    for t in list(ys) + list(xs):
        assert t.is_cuda and t.is_contiguous()
    _ok(LIB.mg_coarse_apply_multi(c_ctx, c_lev, c_y, c_x, k, nrhs, _stream(stream)), ctxs[0])


def mg_set_setup_sweeps(ctx, sweeps):
    _ok(LIB.mg_set_setup_sweeps(ctx, sweeps), ctx)


def _dims(d):
    return (C.c_int * 4)(*[int(v) for v in d])


def mg_cnn_create(nvec, seed=1):
    h = C.c_void_p()
    _ok(LIB.mg_cnn_create(nvec, seed, C.byref(h)))
    return h


def mg_cnn_destroy(net):
    _ok(LIB.mg_cnn_destroy(net))


def mg_cnn_nparams(net) -> int:
    n = C.c_int()
    _ok(LIB.mg_cnn_nparams(net, C.byref(n)))
    return n.value


def mg_cnn_get_params(net, out, which=0, stream=None):
    _ok(LIB.mg_cnn_get_params(net, _ptr(out), out.numel() * 4, which, _stream(stream)))
    return out


def mg_cnn_set_params(net, params, stream=None):
    assert params.dtype == torch.float32
    _ok(LIB.mg_cnn_set_params(net, _ptr(params), params.numel() * 4, _stream(stream)))


def mg_cnn_forward(net, dims, gauge, out, stream=None):
    _ok(LIB.mg_cnn_forward(net, _dims(dims), _ptr(gauge), _ptr(out), _stream(stream)))
    return out


def mg_cnn_loss_grad(net, dims, block, gauge, target, stream=None) -> float:
    loss = C.c_double()
    _ok(LIB.mg_cnn_loss_grad(net, _dims(dims), _dims(block), _ptr(gauge), _ptr(target),
                             C.byref(loss), _stream(stream)))
    return loss.value


def mg_cnn_adam_step(net, lr, stream=None):
    _ok(LIB.mg_cnn_adam_step(net, lr, _stream(stream)))


def mg_fma_peak(prec, stream=None) -> float:
    """Measured FP32 (prec = F32) or FP64 (F64) FMA peak in TFLOP/s."""
    t = C.c_double()
    _ok(LIB.mg_fma_peak(int(prec), C.byref(t), _stream(stream)), None)
    return t.value


def mg_launch_count(ctx) -> int:
    return int(LIB.mg_launch_count(ctx))


def mg_halo_plan(dims, procs, rank):
    """Host-only exchange plan of one rank: dict of per-face lists
    send_to, recv_from, face_offset, face_sites (8 faces, f = 2 mu + s)."""
    arrs = [(C.c_int * 8)() for _ in range(4)]
    _ok(LIB.mg_halo_plan(_dims(dims), _dims(procs), int(rank), *arrs), None)
    names = ("send_to", "recv_from", "face_offset", "face_sites")
    return {k: list(a) for k, a in zip(names, arrs)}


def mg_halo_face_sites(local_dims, mu, side):
    """Host-only: local site indices of one face, in face order."""
    n = 1
    for m, v in enumerate(local_dims):
        if m != mu:
            n *= int(v)
    out = (C.c_int * n)()
    _ok(LIB.mg_halo_face_sites(_dims(local_dims), int(mu), int(side), out), None)
    return list(out)


def mg_halo_create(ctx, level, procs, stream=None):
    h = C.c_void_p()
    _ok(LIB.mg_halo_create(ctx, level, _dims(procs), C.byref(h), _stream(stream)), None)
    return h


def mg_halo_destroy(h):
    _ok(LIB.mg_halo_destroy(h), None)


def mg_halo_info(h):
    nr, ld, hs, hb = C.c_int(), (C.c_int * 4)(), C.c_int(), C.c_size_t()
    _ok(LIB.mg_halo_info(h, C.byref(nr), ld, C.byref(hs), C.byref(hb)), None)
    return dict(nranks=nr.value, local_dims=tuple(ld), halo_sites=hs.value,
                halo_bytes=hb.value)


def mg_halo_scatter(h, rank, local, glob, to_global=False, stream=None):
    _ok(LIB.mg_halo_scatter(h, rank, _ptr(local), _ptr(glob), int(bool(to_global)),
                            _stream(stream)), None)


def mg_halo_pack(h, rank, local, stream=None):
    _ok(LIB.mg_halo_pack(h, rank, _ptr(local), _stream(stream)), None)


def mg_halo_exchange(h, stream=None):
    _ok(LIB.mg_halo_exchange(h, _stream(stream)), None)


def mg_halo_apply(h, rank, y, x, stream=None):
    _ok(LIB.mg_halo_apply(h, rank, _ptr(y), _ptr(x), _stream(stream)), None)


def mg_halo_buffers(h, rank):
    s, r = C.c_void_p(), C.c_void_p()
    _ok(LIB.mg_halo_buffers(h, rank, C.byref(s), C.byref(r)), None)
    return s.value, r.value


def mg_halo_launch_count(h) -> int:
    return int(LIB.mg_halo_launch_count(h))


class Halo:
    """Owner of an mg_halo: coarse level `level` of ctx cut into sub-domains."""

    def __init__(self, ctx, level, procs, stream=None):
        self.h = mg_halo_create(ctx, level, procs, stream)
        info = mg_halo_info(self.h)
        self.nranks, self.local_dims = info["nranks"], info["local_dims"]
        self.halo_sites, self.halo_bytes = info["halo_sites"], info["halo_bytes"]

    def close(self):
        if self.h is not None:
            mg_halo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def scatter(self, rank, local, glob, stream=None):
        mg_halo_scatter(self.h, rank, local, glob, False, stream)

    def gather(self, rank, glob, local, stream=None):
        mg_halo_scatter(self.h, rank, local, glob, True, stream)

    def pack(self, rank, local, stream=None):
        mg_halo_pack(self.h, rank, local, stream)

    def exchange(self, stream=None):
        mg_halo_exchange(self.h, stream)

    def apply(self, rank, y, x, stream=None):
        mg_halo_apply(self.h, rank, y, x, stream)

    def buffers(self, rank):
        return mg_halo_buffers(self.h, rank)

    def launch_count(self):
        return mg_halo_launch_count(self.h)


class Multigrid:
    """Owner of an mg_ctx with the per-level vector shapes at hand."""

    def __init__(self, params: mg_params, gauge: torch.Tensor):
        self.params = params
        self.ctx = mg_create(params, gauge)
        self.levels = [mg_level_info(self.ctx, l) for l in range(params.nlevels)]

    def close(self):
        if self.ctx is not None:
            mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vector(self, level, nrhs=1, dtype=None):
        li = self.levels[level]
        shape = (li["volume"], li["ndof"]) + ((nrhs,) if nrhs > 1 else ())
        return torch.zeros(shape, dtype=dtype or li["dtype"], device="cuda")
