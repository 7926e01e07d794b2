"""Thin Python binding of liblmfmm (include/lmfmm.h): the layered-media FMM of
Cho & Huang (arXiv:1902.08250) on a GB300 GPU.

Argument marshalling only: every step of create/build/apply runs in the CUDA
library.  PyTorch supplies device memory and the current stream.  If the
library cannot be built or loaded, importing this package raises -- there is
no CPU path.

    import torch, paper_1902_08250_gb300 as lm
    med = lm.create_medium(1.0, 1.5, 2.0, 1.0, p=20)
    tree = lm.build_tree(med, x, y)          # x, y: float64 CUDA tensors
    u = lm.apply(tree, q)                    # q: complex128 CUDA tensor [nvec, n] or [n]
    w = lm.apply_adjoint(tree, v)
"""
from __future__ import annotations

import ctypes
import os

from . import _build

HAS_MIXED = True

__all__ = [
    "LMError", "Medium", "Tree", "create_medium", "build_tree", "apply", "apply_adjoint", "apply_grad", "green_apply",
    "sync_status", "Batch", "Cross", "build_cross", "library_path", "FP64", "MIXED", "KERNEL_G", "KERNEL_DG_DD",
]

FP64, MIXED = 0, 1
KERNEL_G, KERNEL_DG_DD = 0, 1
BC = {"transmission": 0, "dirichlet": 1, "neumann": 2, "impedance": 3}
_STATUS = {0: "LM_OK", 1: "LM_EINVAL", 2: "LM_ENOMEM", 3: "LM_ECUDA", 4: "LM_ETIMEOUT", 5: "LM_ENOTSUP"}


class LMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Options(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("depth", ctypes.c_int), ("leaf_target", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_nvec", ctypes.c_int), ("seg_order", ctypes.c_int),
                ("tail_order", ctypes.c_int), ("tail_rays", ctypes.c_int), ("tensor_m2l", ctypes.c_int),
                ("kernel", ctypes.c_int), ("autotune", ctypes.c_int), ("top_bc", ctypes.c_int),
                ("bottom_bc", ctypes.c_int), ("top_alpha", ctypes.c_double), ("bottom_alpha", ctypes.c_double),
                ("adaptive", ctypes.c_int), ("m2l_fp64", ctypes.c_int),
                ("tensor_leaf", ctypes.c_int)]


class _TreeInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("R", ctypes.c_int), ("depth", ctypes.c_int), ("p", ctypes.c_int),
                ("x_origin", ctypes.c_double), ("nleaf", ctypes.c_int64), ("precision", ctypes.c_int),
                ("max_nvec", ctypes.c_int), ("device_bytes", ctypes.c_int64), ("nbox", ctypes.c_int64),
                ("adaptive", ctypes.c_int), ("tensor_leaf", ctypes.c_int)]


def _load():
    path = _build.build()
    L = ctypes.CDLL(path)
    V, P, I, I64, D = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "lm_options_default": (I, [P]),
        "lm_create_medium": (I, [D, D, D, D, P, P]),
        "lm_build_tree": (I, [V, P, P, I64, P, P]),
        "lm_apply": (I, [V, P, I, P, P]),
        "lm_apply_adjoint": (I, [V, P, I, P, P]),
        "lm_apply_grad": (I, [V, P, I, P, P, P, P]),
        "lm_apply_c64": (I, [V, P, I, P, P]),
        "lm_autotune": (I, [V, P, P, P]),
        "lm_apply_adjoint_c64": (I, [V, P, I, P, P]),
        "lm_get_tree_info": (I, [V, P]),
        "lm_tree_export": (I, [V, P, P, P]),
        "lm_list_export": (I, [V, I, I, P, I64, P, P]),
        "lm_box_export": (I, [V, P, I64, P]),
        "lm_adaptive_plan": (I, [P, P, I64, D, I, I, P, P, P, P, I64, P, P, P, P, I64, P, P, I64]),
        "lm_m2l_table_export": (I, [V, I, I, I, I, P, P]),
        "lm_profile_begin": (I, [V, I]),
        "lm_profile_end": (I, [V, P, P, I, P]),
        "lm_peak_probe": (I, [I, I64, P, P]),
        "lm_tree_order_noalloc": (I, [P, P, I64, D, I, P, P, I64, P, P, P]),
        "lm_sync_status": (I, [V, P]),
        "lm_set_poll_limit": (I, [V, I]),
        "lm_misfit_grad_workspace": (I, [V, I, P]),
        "lm_misfit_grad": (I, [V, V, P, P, I, P, P, P, P, P, ctypes.c_size_t, P]),
        "lm_batch_create": (I, [P, I, P, P, P, P, P]),
        "lm_batch_launch": (I, [V, P]),
        "lm_batch_info": (I, [V, P, P]),
        "lm_build_cross": (I, [V, P, P, I64, P, P, I64, P, P]),
        "lm_cross_apply": (I, [V, P, I, P, P]),
        "lm_cross_info": (I, [V, P, P, P, P, P]),
        "lm_destroy_cross": (None, [V]),
        "lm_batch_destroy": (None, [V]),
        "lm_destroy_tree": (None, [V]),
        "lm_destroy_medium": (None, [V]),
        "lm_status_string": (ctypes.c_char_p, [I]),
        "lm_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_lib = _load()


def library_path() -> str:
    return _build.LIB


def _check(status):
    if status != 0:
        raise LMError(status, _lib.lm_last_error().decode())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Medium:
    """Three-layer medium (Sec. 3, Example 4) plus FMM options."""

    def __init__(self, handle, k1, k2, k3, d, opts):
        self._h = ctypes.c_void_p(handle)
        self.k1, self.k2, self.k3, self.d = k1, k2, k3, d
        self.options = opts

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lm_destroy_medium(self._h)
            self._h = None


def create_medium(k1, k2, k3, d, *, p=20, depth=-1, leaf_target=48, precision=FP64, max_nvec=16,
                  seg_order=0, tail_order=0, tail_rays=9, tensor_m2l=1, kernel=KERNEL_G,
                  autotune=0, top_bc="transmission", top_alpha=0.0, bottom_bc="transmission",
                  bottom_alpha=0.0, adaptive=False, m2l_fp64=False, tensor_leaf=1) -> Medium:
    """kernel = KERNEL_G applies G; KERNEL_DG_DD applies dG/dd at fixed points.
    autotune = 1 tunes the M2L tile shapes of mixed-precision trees at build time.
    top_bc / bottom_bc: "transmission" (to the outer layer, k1 / k3), or a wall --
    "dirichlet", "neumann", "impedance" (du/dn - i k2 alpha u = 0, alpha = top_alpha /
    bottom_alpha).
    adaptive = True builds adaptive trees (either precision): a box with more than leaf_target points is
    split while its level is below depth (-1 -> 14).
    m2l_fp64 = True runs the FP64 form's M2L, M2M and L2L contractions in IEEE FP64 instead of
    double-float on the FP32 pipes.
    tensor_leaf = 0 keeps the mixed leaf step (S2T and L2T) of 16-vector applies on the CUDA cores."""
    if isinstance(precision, str):
        precision = {"fp64": FP64, "mixed": MIXED}[precision]
    for b in (top_bc, bottom_bc):
        if b not in BC:
            raise ValueError(f"create_medium: unknown boundary kind {b!r} (one of {sorted(BC)})")
    o = _Options(p, depth, leaf_target, precision, max_nvec, seg_order, tail_order, tail_rays, tensor_m2l,
                 kernel, autotune, BC[top_bc], BC[bottom_bc], float(top_alpha), float(bottom_alpha),
                 int(bool(adaptive)), int(bool(m2l_fp64)), int(bool(tensor_leaf)))
    h = ctypes.c_void_p()
    _check(_lib.lm_create_medium(k1, k2, k3, d, ctypes.byref(o), ctypes.byref(h)))
    return Medium(h.value, k1, k2, k3, d, dict(p=p, depth=depth, leaf_target=leaf_target,
                                              precision=precision, max_nvec=max_nvec, seg_order=seg_order,
                                              tail_order=tail_order, tail_rays=tail_rays,
                                              tensor_m2l=tensor_m2l, kernel=kernel, autotune=autotune,
                                              top_bc=top_bc, top_alpha=top_alpha, bottom_bc=bottom_bc,
                                              bottom_alpha=bottom_alpha, adaptive=bool(adaptive),
                                              m2l_fp64=bool(m2l_fp64), tensor_leaf=int(bool(tensor_leaf))))


class Tree:
    """A built tree: points, lists and translation tables on the device."""

    def __init__(self, handle, medium, x=None, y=None):
        self._h = ctypes.c_void_p(handle)
        self.medium = medium
        self.info = self._info()
        self.n = self.info["n"]
        self._x, self._y = x, y   # the caller's coordinate tensors (not copied)
        self._dtree = None

    def autotune(self, stream=None):
        """Tune the M2L tile shape per level (lm_autotune); returns [(choice, ms)] per level:
        choice -1 = no stencil, 0 = tensor cores, r = CUDA cores with r orders per thread."""
        nl = self.info["depth"] + 1
        ch = (ctypes.c_int * nl)()
        ms = (ctypes.c_float * nl)()
        _check(_lib.lm_autotune(self._h, _stream(stream), ch, ms))
        return [(ch[i], ms[i]) for i in range(nl)]

    def d_tree(self):
        """The tree of dG/dd over the same points and options (built once, cached)."""
        if self._dtree is None:
            m = self.medium
            opts = dict(m.options)
            opts["kernel"] = KERNEL_DG_DD
            md = create_medium(m.k1, m.k2, m.k3, m.d, **opts)
            self._dtree = build_tree(md, self._x, self._y)
        return self._dtree

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lm_destroy_tree(self._h)
            self._h = None

    def _info(self):
        i = _TreeInfo()
        _check(_lib.lm_get_tree_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in _TreeInfo._fields_}

    def export(self, stream=None):
        """(perm, leaf_start) as numpy int64 arrays (tree order); for an adaptive tree
        leaf_start has one entry per box (boxes that are not leaves own no points)."""
        import numpy as np

        info = self.info
        perm = np.zeros(self.n, np.int64)
        ls = np.zeros((info["nbox"] if info["adaptive"] else info["nleaf"]) + 1, np.int64)
        _check(_lib.lm_tree_export(self._h, perm.ctypes.data_as(ctypes.c_void_p),
                                   ls.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        return perm, ls

    def boxes(self):
        """Rows (level, column, row, leaf) of every box, in box-id order."""
        import numpy as np

        cnt = ctypes.c_int64()
        _check(_lib.lm_box_export(self._h, None, 0, ctypes.byref(cnt)))
        out = np.zeros((max(cnt.value, 1), 4), np.int64)
        _check(_lib.lm_box_export(self._h, out.ctypes.data_as(ctypes.c_void_p), cnt.value, ctypes.byref(cnt)))
        return out[:cnt.value]

    def list_export(self, which, level=0, stream=None):
        """Rows (target box, term, source box) of the V list of `level` (which=0) or the U list (1)."""
        import numpy as np

        cnt = ctypes.c_int64()
        _check(_lib.lm_list_export(self._h, which, level, None, 0, ctypes.byref(cnt), _stream(stream)))
        out = np.zeros((max(cnt.value, 1), 3), np.int64)
        _check(_lib.lm_list_export(self._h, which, level, out.ctypes.data_as(ctypes.c_void_p), cnt.value,
                                   ctypes.byref(cnt), _stream(stream)))
        return out[:cnt.value]

    def m2l_table(self, level, term, dc, dr, stream=None):
        import numpy as np

        P = self.info["p"]
        out = np.zeros((2 * P + 1, 2 * P + 1), np.complex128)
        _check(_lib.lm_m2l_table_export(self._h, level, term, dc, dr, out.ctypes.data_as(ctypes.c_void_p),
                                        _stream(stream)))
        return out


def adaptive_plan(x, y, d, leaf_target=48, depth=-1):
    """The adaptive tree of build_tree (adaptive=True) planned on the host from numpy
    arrays, without a GPU: ((x_origin, R), boxes [nbox, 4] = (level, column, row, leaf),
    perm, pstart [nbox + 1], V rows, U rows), rows (target box, term, source box)."""
    import numpy as np

    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    if x.shape != y.shape or x.ndim != 1:
        raise ValueError("adaptive_plan: x and y must be 1-D arrays of the same length")
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    x0, R = ctypes.c_double(), ctypes.c_int()
    nb, nv, nu = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    args = (ptr(x), ptr(y), x.size, float(d), int(leaf_target), int(depth))
    _check(_lib.lm_adaptive_plan(*args, ctypes.byref(x0), ctypes.byref(R), ctypes.byref(nb), None, 0, None, None,
                                 ctypes.byref(nv), None, 0, ctypes.byref(nu), None, 0))
    boxes = np.zeros((nb.value, 4), np.int64)
    pstart = np.zeros(nb.value + 1, np.int64)
    perm = np.zeros(x.size, np.int64)
    V = np.zeros((max(nv.value, 1), 3), np.int64)
    U = np.zeros((max(nu.value, 1), 3), np.int64)
    _check(_lib.lm_adaptive_plan(*args, None, None, None, ptr(boxes), nb.value, ptr(perm), ptr(pstart), None,
                                 ptr(V), nv.value, None, ptr(U), nu.value))
    return (x0.value, R.value), boxes, perm, pstart, V[:nv.value], U[:nu.value]


def build_tree(medium: Medium, x, y, stream=None) -> Tree:
    """x, y: contiguous float64 CUDA tensors of the point coordinates."""
    import torch

    for a in (x, y):
        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
            raise ValueError("build_tree: x and y must be contiguous float64 CUDA tensors")
    if x.numel() != y.numel():
        raise ValueError("build_tree: x and y differ in length")
    h = ctypes.c_void_p()
    _check(_lib.lm_build_tree(medium._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                              x.numel(), _stream(stream), ctypes.byref(h)))
    return Tree(h.value, medium, x, y)


def _apply(fn, tree, q, u, stream, fn64=None):
    import torch

    if fn64 is not None and q.dtype == torch.complex64:
        fn = fn64  # complex64 buffers (LM_MIXED trees)
    elif q.dtype != torch.complex128:
        raise ValueError("apply: q must be complex128 (or complex64 on a mixed-precision tree)")
    if not (q.is_cuda and q.is_contiguous()):
        raise ValueError("apply: q must be a contiguous CUDA tensor")
    one = q.dim() == 1
    q2 = q.reshape(1, -1) if one else q
    if q2.shape[-1] != tree.n:
        raise ValueError(f"apply: q has {q2.shape[-1]} points, tree has {tree.n}")
    if u is None:
        u = torch.empty_like(q2)
    _check(fn(tree._h, ctypes.c_void_p(q2.data_ptr()), q2.shape[0], ctypes.c_void_p(u.data_ptr()),
              _stream(stream)))
    return u.reshape(-1) if one else u


def apply(tree: Tree, q, u=None, stream=None):
    """u = G q (Algorithm 1). q: complex128 CUDA tensor [nvec, n] or [n] (complex64 on a
    mixed-precision tree; u then has the same dtype)."""
    return _apply(_lib.lm_apply, tree, q, u, stream, _lib.lm_apply_c64)


def sync_status(tree: Tree, stream=None):
    """Synchronise and raise LMError(LM_ETIMEOUT) if a bounded device wait gave up."""
    _check(_lib.lm_sync_status(tree._h, _stream(stream)))


def set_poll_limit(tree: Tree, limit):
    """Limit the polls of the tensor-core M2L's first operand wait in the tree's next
    16-vector apply (lm_set_poll_limit; 0 gives up at once, < 0 clears)."""
    _check(_lib.lm_set_poll_limit(tree._h, int(limit)))


def apply_adjoint(tree: Tree, v, w=None, stream=None):
    """w = G^H v = conj(G conj(v)) (reciprocity)."""
    return _apply(_lib.lm_apply_adjoint, tree, v, w, stream, _lib.lm_apply_adjoint_c64)


def apply_grad(tree: Tree, q, stream=None, want_u=True):
    """(u, du/dx, du/dy) at the points, sources held fixed (lm_apply_grad; FP64 trees).
    q: complex128 CUDA tensor [nvec, n] or [n]; u is None when want_u is False."""
    import torch

    if not (q.is_cuda and q.dtype == torch.complex128 and q.is_contiguous()):
        raise ValueError("apply_grad: q must be a contiguous complex128 CUDA tensor")
    one = q.dim() == 1
    q2 = q.reshape(1, -1) if one else q
    if q2.shape[-1] != tree.n:
        raise ValueError(f"apply_grad: q has {q2.shape[-1]} points, tree has {tree.n}")
    u = torch.empty_like(q2) if want_u else None
    ux, uy = torch.empty_like(q2), torch.empty_like(q2)
    _check(_lib.lm_apply_grad(tree._h, ctypes.c_void_p(q2.data_ptr()), q2.shape[0],
                              ctypes.c_void_p(u.data_ptr()) if want_u else None, ctypes.c_void_p(ux.data_ptr()),
                              ctypes.c_void_p(uy.data_ptr()), _stream(stream)))
    if one:
        return (u.reshape(-1) if want_u else None), ux.reshape(-1), uy.reshape(-1)
    return u, ux, uy


def _autograd_function():
    import torch

    class _LayeredGreen(torch.autograd.Function):
        """u = G(x, y, d) q.  With g = dL/du (PyTorch's convention for a real L) the
        backward is one lm_misfit_grad call: dL/dq = G^H g, dL/dx_j = Re[conj(g_j) ux(q)_j
        + q_j ux(conj g)_j] and the same in y (target gradient + reciprocity
        G(a, b) = G(b, a)), dL/dd = Re sum_i conj(g_i) (dG/dd q)_i (the dG/dd tree), all
        formed by the library's kernels.  This class only allocates the outputs and the
        workspace and passes pointers."""

        @staticmethod
        def forward(ctx, q, x, y, d, tree):
            ctx.tree = tree
            ctx.one = q.dim() == 1
            ctx.save_for_backward(q)
            return apply(tree, q.contiguous())

        @staticmethod
        def backward(ctx, grad_u):
            (q,) = ctx.saved_tensors
            t = ctx.tree
            g = grad_u.contiguous()
            qc = q.contiguous()
            nvec = 1 if ctx.one else q.shape[0]
            need = ctx.needs_input_grad
            dev = q.device
            gq = torch.empty_like(qc) if need[0] else None
            gx = torch.empty(t.n, dtype=torch.float64, device=dev) if need[1] else None
            gy = torch.empty(t.n, dtype=torch.float64, device=dev) if need[2] else None
            gd = torch.empty((), dtype=torch.float64, device=dev) if need[3] else None
            dt = t.d_tree() if need[3] else None
            ws, nbytes = None, 0
            if need[1] or need[2] or need[3]:
                b = ctypes.c_size_t()
                _check(_lib.lm_misfit_grad_workspace(t._h, nvec, ctypes.byref(b)))
                nbytes = b.value
                ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)

            def ptr(a):
                return None if a is None else ctypes.c_void_p(a.data_ptr())

            _check(_lib.lm_misfit_grad(t._h, dt._h if dt is not None else None, ptr(qc), ptr(g), nvec, ptr(gq),
                                       ptr(gx), ptr(gy), ptr(gd), ptr(ws), nbytes, _stream(None)))
            return gq, gx, gy, gd, None

    return _LayeredGreen


_LG = None


def green_apply(tree: Tree, q, x=None, y=None, d=None):
    """Differentiable u = G q (PyTorch autograd).

    Gradients flow to the complex densities q (adjoint apply, Sec. 3
    reciprocity: G^H v = conj(G conj(v))), and, when given, to the point
    coordinates x, y (float64 CUDA tensors holding the values the tree was
    built on) and to the layer thickness d (a 0-dim float64 tensor equal to the
    medium's d).  Coordinate gradients need an FP64 tree."""
    import torch

    global _LG
    if _LG is None:
        _LG = _autograd_function()
    for a, ref in ((x, tree._x), (y, tree._y)):
        if a is not None and a is not ref and not torch.equal(a.detach(), ref):
            raise ValueError("green_apply: x and y must hold the coordinates the tree was built on")
    if d is not None and float(d.detach()) != tree.medium.d:
        raise ValueError("green_apply: d must equal the medium's thickness")
    return _LG.apply(q, x, y, d, tree)


class Batch:
    """Applies of several trees captured into one CUDA graph (lm_batch_create);
    launch() replays them, reading the bound q buffers and writing the u buffers."""

    def __init__(self, trees, qs, us):
        import torch

        if not (len(trees) == len(qs) == len(us)) or not trees:
            raise ValueError("Batch: trees, qs and us must be non-empty and of equal length")
        self.trees, self.qs, self.us = list(trees), list(qs), list(us)   # keep buffers alive
        n = len(trees)
        for t, q, u in zip(trees, qs, us):
            for a in (q, u):
                if not (a.is_cuda and a.dtype in (torch.complex128, torch.complex64) and a.is_contiguous()):
                    raise ValueError("Batch: buffers must be contiguous complex128 or complex64 CUDA tensors")
            if q.shape[-1] != t.n or u.shape != q.shape or u.dtype != q.dtype:
                raise ValueError("Batch: buffer shape or dtype does not match its tree")
        th = (ctypes.c_void_p * n)(*[t._h.value for t in trees])
        qp = (ctypes.c_void_p * n)(*[q.data_ptr() for q in qs])
        up = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
        nv = (ctypes.c_int * n)(*[1 if q.dim() == 1 else q.shape[0] for q in qs])
        c64 = (ctypes.c_int * n)(*[int(q.dtype == torch.complex64) for q in qs])
        h = ctypes.c_void_p()
        _check(_lib.lm_batch_create(th, n, qp, nv, up, c64, ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(_lib.lm_batch_launch(self._h, _stream(stream)))

    def info(self):
        """(kernel launches per launch(), whether one M2L launch serves every tree)."""
        k, j = ctypes.c_int64(), ctypes.c_int()
        _check(_lib.lm_batch_info(self._h, ctypes.byref(k), ctypes.byref(j)))
        return k.value, bool(j.value)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lm_batch_destroy(self._h)
            self._h = None


class Cross:
    """Cross-layer operator (Example 4 as printed): layer-1 sources -> middle-layer targets."""

    def __init__(self, handle, medium, ns, nt):
        self._h = ctypes.c_void_p(handle)
        self.medium, self.ns, self.nt = medium, ns, nt
        R, L, x0 = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(_lib.lm_cross_info(self._h, None, None, ctypes.byref(R), ctypes.byref(L), ctypes.byref(x0)))
        self.info = {"R": R.value, "depth": L.value, "x_origin": x0.value, "ns": ns, "nt": nt}

    def apply(self, q, u=None, stream=None):
        """u = (g_2^t + g_2^b) q: q complex128 CUDA [nvec, ns] or [ns] -> [nvec, nt] or [nt]."""
        import torch

        if not (q.is_cuda and q.dtype == torch.complex128 and q.is_contiguous()):
            raise ValueError("Cross.apply: q must be a contiguous complex128 CUDA tensor")
        one = q.dim() == 1
        q2 = q.reshape(1, -1) if one else q
        if q2.shape[-1] != self.ns:
            raise ValueError(f"Cross.apply: q has {q2.shape[-1]} sources, the operator has {self.ns}")
        if u is None:
            u = torch.empty((q2.shape[0], self.nt), dtype=torch.complex128, device=q.device)
        _check(_lib.lm_cross_apply(self._h, ctypes.c_void_p(q2.data_ptr()), q2.shape[0],
                                   ctypes.c_void_p(u.data_ptr()), _stream(stream)))
        return u.reshape(-1) if one else u

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.lm_destroy_cross(self._h)
            self._h = None


def build_cross(medium: Medium, xs, ys, xt, yt, stream=None) -> Cross:
    """Sources (xs, ys), 0 < ys < d, in layer 1; targets (xt, yt), -d < yt < 0; float64 CUDA tensors."""
    import torch

    for a in (xs, ys, xt, yt):
        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
            raise ValueError("build_cross: coordinates must be contiguous float64 CUDA tensors")
    if xs.numel() != ys.numel() or xt.numel() != yt.numel():
        raise ValueError("build_cross: coordinate arrays differ in length")
    h = ctypes.c_void_p()
    _check(_lib.lm_build_cross(medium._h, ctypes.c_void_p(xs.data_ptr()), ctypes.c_void_p(ys.data_ptr()),
                               xs.numel(), ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(yt.data_ptr()),
                               xt.numel(), _stream(stream), ctypes.byref(h)))
    return Cross(h.value, medium, xs.numel(), xt.numel())
