"""Python binding of the nsp C ABI (include/nsp.h): argument marshalling only.

Every numerical step runs in the CUDA library ``libnsp.so`` built in-tree by
``paper_2101_12164_gb300.build``; there is no CPU fallback. Loading fails loudly when the
library is missing. PyTorch is used only for device memory and the current CUDA stream.

Function names follow the C ABI (``nsp_build``, ``nsp_apply``, ``nsp_solve`` ...); the
``Handle`` class wraps a built preconditioner.
"""

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnsp.so")

NSP_FP64, NSP_FP32 = 0, 1
NSP_OUTER_AUTO, NSP_OUTER_SCHUR, NSP_OUTER_FULL = 0, 1, 2
NSP_VARIANT_M2, NSP_VARIANT_M2_ADEF, NSP_VARIANT_M3, NSP_VARIANT_M3_ADEF, NSP_VARIANT_M1 = 0, 1, 2, 3, 4
NSP_FORM_SGAMMA, NSP_FORM_SI = 0, 1
STATUS = {0: "NSP_OK", 1: "NSP_ERR_INVALID_ARG", 2: "NSP_ERR_NOT_DBBD", 3: "NSP_ERR_NOT_SPD",
          4: "NSP_ERR_BREAKDOWN", 5: "NSP_ERR_NOT_CONVERGED", 6: "NSP_ERR_TIMEOUT",
          7: "NSP_ERR_CUDA", 8: "NSP_ERR_OOM", 9: "NSP_ERR_UNSUPPORTED"}
EXPORTS = ["nsp_default_params", "nsp_build", "nsp_rebuild", "nsp_apply", "nsp_solve",
           "nsp_schur_apply", "nsp_factor_solve", "nsp_get_basis", "nsp_get_intermediate",
           "nsp_get_factor", "nsp_get_info", "nsp_destroy", "nsp_status_string", "nsp_last_error", "nsp_gaussian",
           "nsp_analyze", "nsp_kernel_launches", "nsp_schur_apply_noalloc", "nsp_build_batched",
           "nsp_solve_batched", "nsp_net_num_params", "nsp_net_create", "nsp_net_set_params",
           "nsp_net_get", "nsp_net_forward", "nsp_net_loss_grad", "nsp_net_zero_grad",
           "nsp_net_adam_step", "nsp_net_sketch", "nsp_net_destroy", "nsp_check_timeout_path",
           "nsp_gram_work_bytes", "nsp_gram", "nsp_gram_compensated",
           "nsp_block_update_work_bytes", "nsp_block_update"]


class NspError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s" % (where, STATUS.get(status, status)))


class nsp_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int32)]


class nsp_partition(C.Structure):
    _fields_ = [("nblocks", C.c_int32), ("part", C.c_void_p), ("perm", C.c_void_p)]


class nsp_params(C.Structure):
    _fields_ = [("k", C.c_int32), ("p", C.c_int32), ("eps_inner", C.c_double),
                ("eps_trunc_rel", C.c_double), ("drop_tol", C.c_double),
                ("max_inner_it", C.c_int32), ("seed", C.c_uint64), ("sketch", C.c_void_p),
                ("precision", C.c_int32), ("outer_form", C.c_int32), ("inner_form", C.c_int32),
                ("keep_intermediates", C.c_int32), ("stream", C.c_void_p),
                ("variant", C.c_int32), ("q", C.c_int32),
                ("gamma_levels", C.c_int32), ("gamma_nblocks", C.c_int32),
                ("gamma_part", C.c_void_p), ("gamma_k", C.c_int32), ("gamma_p", C.c_int32),
                ("gamma_eps_inner", C.c_double), ("gamma_sketch", C.c_void_p)]


class nsp_net_shape(C.Structure):
    _fields_ = [("d_raw", C.c_int32), ("n_coord", C.c_int32), ("n_freq", C.c_int32),
                ("hidden", C.c_int32), ("s_out", C.c_int32), ("precision", C.c_int32),
                ("mu", C.c_double)]


class nsp_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_interior", C.c_int64), ("n_gamma", C.c_int64),
                ("nblocks", C.c_int32), ("nnz_L_interior", C.c_int64),
                ("nnz_L_gamma", C.c_int64), ("n_supernodes", C.c_int64),
                ("it_inner", C.c_int32), ("inner_active_cols", C.c_int32), ("rank", C.c_int32),
                ("it_pcg", C.c_int32), ("inner_residual", C.c_double),
                ("final_residual", C.c_double), ("pcg_residual", C.c_double),
                ("failed_block", C.c_int32), ("ms_analyze", C.c_double),
                ("ms_factor", C.c_double), ("ms_inner", C.c_double), ("ms_core", C.c_double),
                ("ms_solve", C.c_double), ("it_power", C.c_int32),
                ("lambda_min_est", C.c_double), ("lambda_max_est", C.c_double),
                ("kappa_est", C.c_double), ("n_gamma2", C.c_int64),
                ("it_inner_gamma", C.c_int32), ("rank_gamma", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """The loaded CUDA library (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnsp.so is not built: run paper_2101_12164_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        sig = {
            "nsp_default_params": (None, [C.POINTER(nsp_params)]),
            "nsp_build": (C.c_int, [C.POINTER(nsp_csr), C.POINTER(nsp_partition),
                                    C.POINTER(nsp_params), C.POINTER(P)]),
            "nsp_rebuild": (C.c_int, [P, P, C.c_int32, C.POINTER(nsp_params)]),
            "nsp_apply": (C.c_int, [P, P, P]),
            "nsp_solve": (C.c_int, [P, P, P, C.c_double, C.c_int32, C.POINTER(nsp_info)]),
            "nsp_schur_apply": (C.c_int, [P, P, P, C.c_int32]),
            "nsp_factor_solve": (C.c_int, [P, C.c_int32, P, P, C.c_int32]),
            "nsp_get_basis": (C.c_int, [P, P, P, C.POINTER(C.c_int32)]),
            "nsp_get_intermediate": (C.c_int, [P, C.c_int32, P]),
            "nsp_get_factor": (C.c_int, [P, C.c_int32, P, P, C.c_int64]),
            "nsp_get_info": (C.c_int, [P, C.POINTER(nsp_info)]),
            "nsp_destroy": (C.c_int, [P]),
            "nsp_status_string": (C.c_char_p, [C.c_int]),
            "nsp_last_error": (C.c_char_p, []),
            "nsp_gaussian": (C.c_int, [C.c_uint64, C.c_int64, P, P]),
            "nsp_analyze": (C.c_int, [C.POINTER(nsp_csr), C.POINTER(nsp_partition),
                                      C.POINTER(nsp_info)]),
            "nsp_kernel_launches": (C.c_int64, []),
            "nsp_schur_apply_noalloc": (C.c_int, [P, P, P, C.c_int32]),
            "nsp_build_batched": (C.c_int, [C.c_int32, P, P, C.POINTER(nsp_params),
                                            C.POINTER(P)]),
            "nsp_solve_batched": (C.c_int, [P, P, P, C.c_double, C.c_int32, P]),
            "nsp_net_num_params": (C.c_int64, [C.POINTER(nsp_net_shape)]),
            "nsp_net_create": (C.c_int, [C.POINTER(nsp_net_shape), P, P, C.POINTER(P)]),
            "nsp_net_set_params": (C.c_int, [P, P]),
            "nsp_net_get": (C.c_int, [P, C.c_int32, P]),
            "nsp_net_forward": (C.c_int, [P, P, C.c_int64, P]),
            "nsp_net_loss_grad": (C.c_int, [P, P, C.c_int64, P, C.c_int32,
                                            C.POINTER(C.c_double)]),
            "nsp_net_zero_grad": (C.c_int, [P]),
            "nsp_net_adam_step": (C.c_int, [P, C.c_double, C.c_double, C.c_double, C.c_double]),
            "nsp_net_sketch": (C.c_int, [P, P, C.c_int64, P, C.POINTER(C.c_int32)]),
            "nsp_net_destroy": (C.c_int, [P]),
            "nsp_check_timeout_path": (C.c_int, [P, C.c_int32, C.POINTER(C.c_int32)]),
            "nsp_gram_work_bytes": (C.c_int64, [C.c_int64, C.c_int32, C.c_int32]),
            "nsp_gram": (C.c_int, [P, P, C.c_int64, C.c_int32, C.c_int32, P, P, P]),
            "nsp_gram_compensated": (C.c_int, [P, P, C.c_int64, C.c_int32, C.c_int32, P, P, P]),
            "nsp_block_update_work_bytes": (C.c_int64, [C.c_int32, C.c_int32]),
            "nsp_block_update": (C.c_int, [P, P, C.c_int64, C.c_int32, C.c_int32, C.c_float, P,
                                           C.c_float, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, where):
    if status != 0:
        msg = lib().nsp_last_error()
        raise NspError(status, where + (" (%s)" % msg.decode() if msg else ""))


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (must be contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    assert x.flags["C_CONTIGUOUS"]
    return x.ctypes.data


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _csr_struct(A, keep):
    """nsp_csr from a scipy CSR matrix (host) or a (rowptr, col, val) triple of CUDA tensors."""
    if isinstance(A, tuple):
        rowptr, col, val = A
        keep += [rowptr, col, val]
        return nsp_csr(int(rowptr.numel() - 1), _ptr(rowptr), _ptr(col), _ptr(val), 1)
    rowptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    col = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    keep += [rowptr, col, val]
    return nsp_csr(A.shape[0], _ptr(rowptr), _ptr(col), _ptr(val), 0)


def _part_struct(part, nblocks, perm, keep):
    part = np.ascontiguousarray(part, dtype=np.int32)
    keep.append(part)
    pp = None
    if perm is not None:
        perm = np.ascontiguousarray(perm, dtype=np.int64)
        keep.append(perm)
        pp = _ptr(perm)
    return nsp_partition(int(nblocks), _ptr(part), pp)


def nsp_default_params():
    p = nsp_params()
    lib().nsp_default_params(C.byref(p))
    return p


def make_params(k=16, p=10, eps_inner=0.1, eps_trunc_rel=1e-10, drop_tol=None,
                max_inner_it=500, seed=210112164, sketch=None, precision="fp32",
                outer_form="auto", keep_intermediates=False, stream=None, keep=None,
                variant="m2", q=0, inner_form="s_gamma", gamma_part=None, gamma_nblocks=0,
                gamma_k=16, gamma_p=8, gamma_eps_inner=0.1, gamma_sketch=None):
    prm = nsp_default_params()
    prm.k, prm.p = int(k), int(p)
    prm.eps_inner, prm.eps_trunc_rel = float(eps_inner), float(eps_trunc_rel)
    prm.precision = {"fp64": NSP_FP64, "fp32": NSP_FP32}[precision]
    prm.drop_tol = float(drop_tol if drop_tol is not None else
                         (1e-12 if precision == "fp64" else 1e-6))
    prm.max_inner_it = int(max_inner_it)
    prm.seed = int(seed)
    prm.outer_form = {"auto": NSP_OUTER_AUTO, "schur": NSP_OUTER_SCHUR,
                      "full": NSP_OUTER_FULL}[outer_form]
    prm.keep_intermediates = 1 if keep_intermediates else 0
    prm.variant = {"m2": NSP_VARIANT_M2, "m2_adef": NSP_VARIANT_M2_ADEF, "m3": NSP_VARIANT_M3,
                   "m3_adef": NSP_VARIANT_M3_ADEF, "m1": NSP_VARIANT_M1}[variant]
    prm.q = int(q)
    prm.inner_form = {"s_gamma": NSP_FORM_SGAMMA, "s_i": NSP_FORM_SI}[inner_form]
    if sketch is not None:
        if hasattr(sketch, "data_ptr"):   # device tensor: passed through (float64, contiguous)
            if str(sketch.dtype) != "torch.float64" or not sketch.is_contiguous():
                raise ValueError("a device sketch must be a contiguous float64 tensor")
            sk = sketch
        else:
            sk = np.ascontiguousarray(sketch, dtype=np.float64)
        if keep is not None:
            keep.append(sk)
        prm.sketch = _ptr(sk)
    # recursive A_G: its own DBBD split (labels in the caller's Gamma order) and M2' settings
    if gamma_part is not None:
        gp = np.ascontiguousarray(gamma_part, dtype=np.int32)
        if keep is not None:
            keep.append(gp)
        prm.gamma_levels, prm.gamma_nblocks = 1, int(gamma_nblocks)
        prm.gamma_part = _ptr(gp)
    if gamma_sketch is not None:
        gs = np.ascontiguousarray(gamma_sketch, dtype=np.float64)
        if gamma_part is not None:
            rows = int((np.asarray(gamma_part) < 0).sum())
            if gs.size < rows * (int(gamma_k) + int(gamma_p)):
                raise ValueError("gamma_sketch holds %d values; the build reads %d x %d"
                                 % (gs.size, rows, int(gamma_k) + int(gamma_p)))
        if keep is not None:
            keep.append(gs)
        prm.gamma_sketch = _ptr(gs)
    prm.gamma_k, prm.gamma_p = int(gamma_k), int(gamma_p)
    prm.gamma_eps_inner = float(gamma_eps_inner)
    prm.stream = _stream() if stream is None else stream
    return prm


def _check_sketch(kw, n_gamma, n_interior):
    """The library copies rows x (k + p) doubles from a caller sketch (rows = n_Gamma, or
    n_interior for the M3 variants); refuse a smaller buffer before the copy could read past
    its end."""
    sk = kw.get("sketch")
    if sk is None:
        return
    s = int(kw.get("k", 16)) + int(kw.get("p", 10))
    rows = n_interior if kw.get("variant", "m2") in ("m3", "m3_adef") else n_gamma
    size = int(sk.numel()) if hasattr(sk, "numel") else int(np.size(sk))
    if size < rows * s:
        raise ValueError("sketch holds %d values; the build reads %d x %d" % (size, rows, s))


def nsp_build(A, part, nblocks, perm=None, **kw):
    """Build M2 (Algorithm 2) for A; returns a Handle. See make_params for keywords."""
    pa = np.asarray(part)
    _check_sketch(kw, int((pa < 0).sum()), int((pa >= 0).sum()))
    keep = []
    csr = _csr_struct(A, keep)
    ps = _part_struct(part, nblocks, perm, keep)
    prm = make_params(keep=keep, **kw)
    h = C.c_void_p()
    _check(lib().nsp_build(C.byref(csr), C.byref(ps), C.byref(prm), C.byref(h)), "nsp_build")
    return Handle(h, prm, keep)


def nsp_build_batched(mats, **kw):
    """Build one handle for a batch of matrices: mats = [(A, part, nblocks), ...]."""
    _check_sketch(kw, sum(int((np.asarray(pt) < 0).sum()) for _, pt, _ in mats),
                  sum(int((np.asarray(pt) >= 0).sum()) for _, pt, _ in mats))
    keep = []
    csrs = (nsp_csr * len(mats))()
    parts = (nsp_partition * len(mats))()
    for i, (A, part, nb) in enumerate(mats):
        csrs[i] = _csr_struct(A, keep)
        parts[i] = _part_struct(part, nb, None, keep)
    prm = make_params(keep=keep, **kw)
    h = C.c_void_p()
    _check(lib().nsp_build_batched(len(mats), csrs, parts, C.byref(prm), C.byref(h)),
           "nsp_build_batched")
    hd = Handle(h, prm, keep)
    hd.batch = len(mats)
    return hd


class SketchNet:
    """The learned sketch proposal (nsp_net_* calls): raw node attributes -> sketch rows."""

    def __init__(self, theta0, d_raw, n_coord, n_freq, hidden, s_out, precision="fp32",
                 mu=1e-2, stream=None):
        self.shape = nsp_net_shape(int(d_raw), int(n_coord), int(n_freq), int(hidden), int(s_out),
                                   NSP_FP64 if precision == "fp64" else NSP_FP32, float(mu))
        self.num_params = int(lib().nsp_net_num_params(C.byref(self.shape)))
        if self.num_params < 0:
            raise NspError(1, "nsp_net_num_params")
        th = np.ascontiguousarray(theta0, dtype=np.float64)
        if th.size != self.num_params:
            raise ValueError("theta0 has %d entries, the network %d" % (th.size, self.num_params))
        if stream is None:
            stream = _stream()
        self._h = C.c_void_p()
        _check(lib().nsp_net_create(C.byref(self.shape), _ptr(th), C.c_void_p(stream),
                                    C.byref(self._h)), "nsp_net_create")

    def _handle(self):
        if not self._h:
            raise RuntimeError("network destroyed")
        return self._h

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        _check(lib().nsp_net_set_params(self._handle(), _ptr(th)), "nsp_net_set_params")

    def get(self, what=0):
        out = np.zeros(self.num_params)
        _check(lib().nsp_net_get(self._handle(), int(what), _ptr(out)), "nsp_net_get")
        return out

    def params(self):
        return self.get(0)

    def grad(self):
        return self.get(1)

    def forward(self, attrs, G):
        n = attrs.shape[0]
        _check(lib().nsp_net_forward(self._handle(), _ptr(attrs), n, _ptr(G)), "nsp_net_forward")
        return G

    def loss_grad(self, attrs, U, want_loss=True):
        loss = C.c_double(0.0)
        _check(lib().nsp_net_loss_grad(self._handle(), _ptr(attrs), attrs.shape[0], _ptr(U),
                                       U.shape[1], C.byref(loss) if want_loss else None),
               "nsp_net_loss_grad")
        return loss.value if want_loss else None

    def zero_grad(self):
        _check(lib().nsp_net_zero_grad(self._handle()), "nsp_net_zero_grad")

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().nsp_net_adam_step(self._handle(), float(lr), float(beta1), float(beta2),
                                       float(eps)), "nsp_net_adam_step")

    def sketch(self, attrs, G, check=True):
        """Inference into G (n x s_out doubles). With check, G is orthonormalized and the
        return value says whether the proposal had full rank; without, G is the raw output."""
        ok = C.c_int32(0)
        _check(lib().nsp_net_sketch(self._handle(), _ptr(attrs), attrs.shape[0], _ptr(G),
                                    C.byref(ok) if check else None), "nsp_net_sketch")
        return bool(ok.value) if check else None

    def destroy(self):
        if self._h:
            lib().nsp_net_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def nsp_analyze(A, part, nblocks, perm=None):
    """Host-only validation and symbolic analysis; returns nsp_info as a dict."""
    keep = []
    csr = _csr_struct(A, keep)
    ps = _part_struct(part, nblocks, perm, keep)
    info = nsp_info()
    _check(lib().nsp_analyze(C.byref(csr), C.byref(ps), C.byref(info)), "nsp_analyze")
    return info.as_dict()


def nsp_kernel_launches():
    return int(lib().nsp_kernel_launches())


def _status_word(work, nbytes):
    """The device status word the dense-product calls leave in the last 8 bytes of work."""
    import torch
    w = work.view(torch.uint8)[nbytes - 256:nbytes - 248].cpu()
    return int(w.view(torch.int32)[0])


def nsp_gram(X, Y, C, work=None, compensated=False):
    """C = X^T Y (X n x s1, Y n x s2 float32 CUDA tensors, C s1 x s2 float64): on the tensor
    cores, or with compensated FP32 sums (compensated=True, the Nyström core's Grams).
    Synchronizes and checks the kernel's status word."""
    import torch
    n, s1 = X.shape
    s2 = Y.shape[1]
    nb = lib().nsp_gram_work_bytes(n, s1, s2)
    if nb < 0:
        raise NspError(1, "nsp_gram_work_bytes")
    if work is None or work.numel() * work.element_size() < nb:
        work = torch.empty(nb, dtype=torch.uint8, device=X.device)
    fn = lib().nsp_gram_compensated if compensated else lib().nsp_gram
    _check(fn(_ptr(X), _ptr(Y), n, s1, s2, _ptr(C), _ptr(work), _stream()), "nsp_gram")
    torch.cuda.synchronize()
    if _status_word(work, nb) != 0:
        raise NspError(6, "nsp_gram: a bounded device wait ran out")
    return C


def nsp_block_update(A, M, Out, scale=1.0, Cin=None, beta=0.0, work=None):
    """Out = scale * A M + beta * Cin on the tensor cores (A n x s1 float32, M s1 x s2
    float64, Out / Cin n x s2 float32 CUDA tensors). Synchronizes and checks the status."""
    import torch
    n, s1 = A.shape
    s2 = M.shape[1]
    nb = lib().nsp_block_update_work_bytes(s1, s2)
    if nb < 0:
        raise NspError(1, "nsp_block_update_work_bytes")
    if work is None or work.numel() * work.element_size() < nb:
        work = torch.empty(nb, dtype=torch.uint8, device=A.device)
    _check(lib().nsp_block_update(_ptr(A), _ptr(M), n, s1, s2, scale,
                                  _ptr(Cin) if Cin is not None else None, beta, _ptr(Out),
                                  _ptr(work), _stream()), "nsp_block_update")
    torch.cuda.synchronize()
    if _status_word(work, nb) != 0:
        raise NspError(6, "nsp_block_update: a bounded device wait ran out")
    return Out


def nsp_gaussian(seed, count, out):
    _check(lib().nsp_gaussian(int(seed), int(count), _ptr(out), _stream()), "nsp_gaussian")
    return out


class Handle:
    """A built Nyström–Schur preconditioner (owns device memory until destroyed)."""

    def __init__(self, h, prm, keep):
        self._h = h
        self.prm = prm
        self._keep = keep
        self.dtype_name = "float64" if prm.precision == NSP_FP64 else "float32"
        self.batch = 0

    def _handle(self):
        if self._h is None or not self._h.value:
            raise RuntimeError("handle destroyed")
        return self._h

    def info(self):
        inf = nsp_info()
        _check(lib().nsp_get_info(self._handle(), C.byref(inf)), "nsp_get_info")
        return inf.as_dict()

    def rebuild(self, val, on_device=True, **kw):
        keep = []
        prm = make_params(keep=keep, **kw) if kw else None
        if prm is not None:
            prm.stream = self.prm.stream
            prm.gamma_levels = self.prm.gamma_levels   # the A_G split is fixed at the build
        st = lib().nsp_rebuild(self._handle(), _ptr(val), 1 if on_device else 0,
                               C.byref(prm) if prm is not None else None)
        _check(st, "nsp_rebuild")

    def apply(self, r, z):
        _check(lib().nsp_apply(self._handle(), _ptr(r), _ptr(z)), "nsp_apply")
        return z

    def solve(self, b, x, rtol=1e-8, maxit=500, allow_not_converged=False):
        inf = nsp_info()
        st = lib().nsp_solve(self._handle(), _ptr(b), _ptr(x), float(rtol), int(maxit),
                             C.byref(inf))
        if not (st == 0 or (allow_not_converged and st == 5)):
            _check(st, "nsp_solve")
        return inf.as_dict()

    def solve_batched(self, b, x, rtol=1e-8, maxit=500, allow_not_converged=False):
        infos = (nsp_info * self.batch)()
        st = lib().nsp_solve_batched(self._handle(), _ptr(b), _ptr(x), float(rtol), int(maxit),
                                     infos)
        if not (st == 0 or (allow_not_converged and st == 5)):
            _check(st, "nsp_solve_batched")
        return [infos[i].as_dict() for i in range(self.batch)]

    def check_timeout_path(self, max_spins=1 << 14):
        """Status a sweep with unreachable dependencies reports (see nsp_check_timeout_path)."""
        obs = C.c_int32(-1)
        _check(lib().nsp_check_timeout_path(self._handle(), int(max_spins), C.byref(obs)),
               "nsp_check_timeout_path")
        return obs.value

    def schur_apply(self, X, Y):
        s = 1 if X.dim() == 1 else X.shape[1]
        _check(lib().nsp_schur_apply(self._handle(), _ptr(X), _ptr(Y), int(s)), "nsp_schur_apply")
        return Y

    def schur_apply_noalloc(self, X, Y):
        """nsp_schur_apply_noalloc: same result as schur_apply, no device allocation."""
        s = 1 if X.dim() == 1 else X.shape[1]
        _check(lib().nsp_schur_apply_noalloc(self._handle(), _ptr(X), _ptr(Y), int(s)),
               "nsp_schur_apply_noalloc")
        return Y

    def factor_solve(self, which, B, X):
        s = 1 if B.dim() == 1 else B.shape[1]
        _check(lib().nsp_factor_solve(self._handle(), int(which), _ptr(B), _ptr(X), int(s)),
               "nsp_factor_solve")
        return X

    def get_basis(self):
        inf = self.info()
        nG, k = inf["n_gamma"], self.prm.k
        if self.batch:
            # batched handle: all k columns; Sigma per matrix (batch x k)
            Z = np.zeros((nG, k))
            S = np.zeros((self.batch, k))
            r = C.c_int32()
            _check(lib().nsp_get_basis(self._handle(), _ptr(Z), _ptr(S), C.byref(r)),
                   "nsp_get_basis")
            return Z, S
        Z = np.zeros((nG, k))
        S = np.zeros(k)
        r = C.c_int32()
        _check(lib().nsp_get_basis(self._handle(), _ptr(Z), _ptr(S), C.byref(r)), "nsp_get_basis")
        r = r.value
        return np.ascontiguousarray(Z.ravel()[: nG * r].reshape(nG, r)), S[:r]

    def get_intermediate(self, which):
        inf = self.info()
        nG = inf["n_gamma"]
        cols = inf["rank"] if which == 3 else self.prm.k + self.prm.p
        out = np.zeros((nG, max(cols, 1)))
        _check(lib().nsp_get_intermediate(self._handle(), int(which), _ptr(out)),
               "nsp_get_intermediate")
        return out[:, :cols]

    def get_factor(self, block, n_b):
        """(order, L): elimination order (indices in A) and dense lower factor of a block."""
        order = np.zeros(n_b, dtype=np.int64)
        Lf = np.zeros(n_b * n_b)
        _check(lib().nsp_get_factor(self._handle(), int(block), _ptr(order), _ptr(Lf),
                                    int(n_b)), "nsp_get_factor")
        return order, Lf.reshape(n_b, n_b).T.copy()   # column-major -> [row, col]

    def destroy(self):
        if self._h is not None and self._h.value:
            lib().nsp_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
