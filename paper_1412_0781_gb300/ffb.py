"""ctypes binding of ``libffb.so`` (declared in ``include/ffb.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors must be contiguous CUDA tensors of the stated dtype; the
binding passes their device pointers and the current torch stream.  There is
no CPU path: if the library cannot be loaded an ``ImportError`` is raised.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffb.so")

FFB_OK = 0
STATUS = {0: "FFB_OK", -1: "FFB_ERR_ARG", -2: "FFB_ERR_CUDA", -3: "FFB_ERR_OOM",
          -4: "FFB_ERR_NONFINITE", -5: "FFB_ERR_NOT_CONVERGED", -6: "FFB_ERR_TIMEOUT",
          -7: "FFB_ERR_STATE", -8: "FFB_ERR_UNSUPPORTED"}
PRECISION = {"fp32": 0, "bf16": 1, "bf16x3": 2, "tf32": 3, "tf32x3": 4}
DENOISE = {"topk": 0, "mp_wiener": 1, "all": 2, "mp_hard": 3}

# every symbol declared in include/ffb.h, with (restype, argtypes)
_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_pi = ctypes.POINTER(ctypes.c_int)
_pd = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "ffb_plan": (_i, [ctypes.POINTER(_vp), _i, _d, _d, _d, _i, _vp]),
    "ffb_plan_destroy": (_i, [_vp]),
    "ffb_plan_info": (_i, [_vp, _pi]),
    "ffb_plan_sizes": (_i, [_vp, _pi, _pi]),
    "ffb_plan_tables": (_i, [_vp, _pd, _pd, _pd, _pd]),
    "ffb_set_precision": (_i, [_vp, _i]),
    "ffb_set_wait_budget": (_i, [_vp, ctypes.c_longlong]),
    "ffb_polar": (_i, [_vp, _vp, _i64, _vp, _vp]),
    "ffb_polar_noalloc": (_i, [_vp, _vp, _i64, _vp, _vp]),
    "ffb_expand": (_i, [_vp, _vp, _i64, _vp, _vp]),
    "ffb_expand_adjoint": (_i, [_vp, _vp, _i64, _vp, _vp]),
    "ffb_covariance": (_i, [_vp, _vp, _i64, _i, _vp]),
    "ffb_cov_get": (_i, [_vp, _vp, _vp, _vp]),
    "ffb_expand_cov_host": (_i, [_vp, _vp, _i64, _i, _vp, _vp, _vp]),
    "ffb_ringdft_table": (_i, [_i, _i, _vp, _vp]),
    "ffb_cov_export": (_i, [_vp, _pd, _vp]),
    "ffb_cov_merge": (_i, [_i, _pi, _i, _pd, _pd]),
    "ffb_cov_import": (_i, [_vp, _pd, _vp]),
    "ffb_eig": (_i, [_vp, _vp, _vp, _vp]),
    "ffb_eig_blocks": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "ffb_radial_eigenfunctions": (_i, [_vp, _vp, _vp]),
    "ffb_eigenimages": (_i, [_vp, _i, _pi, _pi, _vp, _vp]),
    "ffb_select": (_i, [_vp, _i, _i, _d, _i64, _pd, _vp]),
    "ffb_filter": (_i, [_vp, _vp, _i64, _vp, _i, _vp]),
    "ffb_weight": (_i, [_vp, _vp, _i64, _vp, _vp]),
    "ffb_denoise": (_i, [_vp, _vp, _i64, _i, _i, _d, _vp, _vp]),
    "ffb_sync": (_i, [_vp, _vp]),
    "ffb_profile": (_i, [_vp, _i]),
    "ffb_profile_read": (_i, [_vp, _pd, ctypes.POINTER(ctypes.c_int64)]),
    "ffb_launch_count": (_i64, [_vp]),
    "ffb_estimate_support": (_i, [_vp, _vp, _i64, _d, _d, _pd, _pd, _pd, _vp]),
    "ffb_svd": (_i, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "ffb_invariants": (_i, [_vp, _vp, _i64, _i, _pi, _vp, _i, _pi, _vp, _vp]),
    "ffb_group_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp), _vp]),
    "ffb_group_destroy": (_i, [_vp]),
    "ffb_group_expand_cov": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(_vp), _i, _vp]),
    "ffb_group_covariance": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int64), _i, _vp]),
    "ffb_group_sync": (_i, [_vp, _vp]),
    "ffb_group_info": (_i, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "ffb_group_quad_tuning": (_i, [_vp, _i, _pi, _pi, ctypes.POINTER(ctypes.c_float)]),
    "ffb_group_tuning": (_i, [_vp, _i, _pi, _pi, _pi, ctypes.POINTER(ctypes.c_float)]),
    "ffb_interp_units": (_i, [_i, _i, _d, _i, _i, _pd, ctypes.POINTER(ctypes.c_int64), _vp, _pi]),
    "ffb_tile_units": (_i, [_i, _i, _d, _i, _i, _pd, ctypes.POINTER(ctypes.c_int64), _vp, _pi, _pi]),
    "ffb_strerror": (ctypes.c_char_p, [_i]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libffb.so once and declare its signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libffb.so not built (run __graft_entry__.build()): " + path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def interp_units(N, w, beta, n_theta, xi):
    """Host-only: the shared-memory grid path's interpolation table for radii
    ``xi`` (see ffb_interp_units).  Returns (records float32 (blocks, F, GU,
    4), blocks int32 (blocks, 2), (blocks of half 0, blocks of half 1), MH,
    SLD, nodes per unit at most)."""
    import numpy as np
    x = np.ascontiguousarray(xi, dtype=np.float64)
    cnt = (ctypes.c_int64 * 9)()
    lib = load()
    _check(lib.ffb_interp_units(int(N), int(w), float(beta), len(x), int(n_theta), x.ctypes.data_as(_pd), cnt,
                                None, None), "ffb_interp_units")
    rec = np.zeros(4 * cnt[0], dtype=np.float32)
    blk = np.zeros(2 * cnt[1], dtype=np.int32)
    _check(lib.ffb_interp_units(int(N), int(w), float(beta), len(x), int(n_theta), x.ctypes.data_as(_pd), cnt,
                                rec.ctypes.data_as(ctypes.c_void_p), blk.ctypes.data_as(_pi)),
           "ffb_interp_units")
    gu = int(cnt[4])
    return (rec.reshape(int(cnt[1]), int(cnt[7]), gu, 4), blk.reshape(-1, 2), (int(cnt[2]), int(cnt[3])),
            int(cnt[5]), int(cnt[6]), int(cnt[8]))


def ringdft_table(n_theta, k_max):
    """Host-only: the tensor-core ring DFT's tables (see ffb_ringdft_table):
    (hi, lo) float32 arrays of shape (2, 192, n_theta/2)."""
    import numpy as np
    hi = np.zeros((2, 192, n_theta // 2), dtype=np.float32)
    lo = np.zeros_like(hi)
    _check(load().ffb_ringdft_table(int(n_theta), int(k_max), hi.ctypes.data_as(ctypes.c_void_p),
                                    lo.ctypes.data_as(ctypes.c_void_p)), "ffb_ringdft_table")
    return hi, lo


def tile_units(N, w, beta, n_theta, xi):
    """Host-only: the separate-kernel path's tile interpolation table for
    radii ``xi`` (see ffb_tile_units).  Returns (records float32 (blocks, F,
    GU, 4), blocks int32 (blocks, 4), node lists int32, dict of the tile
    geometry: TR, TC, RS, CS, pitch)."""
    import numpy as np
    x = np.ascontiguousarray(xi, dtype=np.float64)
    cnt = (ctypes.c_int64 * 9)()
    lib = load()
    _check(lib.ffb_tile_units(int(N), int(w), float(beta), len(x), int(n_theta), x.ctypes.data_as(_pd), cnt,
                              None, None, None), "ffb_tile_units")
    nb, nn, F, GU = int(cnt[0]), int(cnt[1]), int(cnt[2]), int(cnt[3])
    rec = np.zeros(nb * F * GU * 4, dtype=np.float32)
    blk = np.zeros(4 * nb, dtype=np.int32)
    nodes = np.zeros(max(nn, 1), dtype=np.int32)
    _check(lib.ffb_tile_units(int(N), int(w), float(beta), len(x), int(n_theta), x.ctypes.data_as(_pd), cnt,
                              rec.ctypes.data_as(ctypes.c_void_p), blk.ctypes.data_as(_pi),
                              nodes.ctypes.data_as(_pi)), "ffb_tile_units")
    geo = {"TR": int(cnt[4]), "TC": int(cnt[5]), "RS": int(cnt[6]), "CS": int(cnt[7]), "pitch": int(cnt[8])}
    return rec.reshape(nb, F, GU, 4), blk.reshape(nb, 4), nodes[:nn], geo


def cov_merge(p, states):
    """Host-only pooling of covariance states (rows of ``states``) for block
    sizes ``p`` (list of p_k); see ffb_cov_merge."""
    import numpy as np
    st = np.ascontiguousarray(states, dtype=np.float64)
    pk = (ctypes.c_int * len(p))(*p)
    out = np.zeros(st.shape[-1])
    _check(load().ffb_cov_merge(len(p) - 1, pk, int(st.shape[0]), st.ctypes.data_as(_pd),
                                out.ctypes.data_as(_pd)), "ffb_cov_merge")
    return out


class FFBError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status),
                                          load().ffb_strerror(status).decode()))


def _check(status, where):
    if status != FFB_OK:
        raise FFBError(status, where)


def _ptr(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t, dtype, name):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a host (CPU) tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """Owns an ffb plan (device tables, scratch, covariance accumulator)."""

    def __init__(self, L, c=0.5, R=None, eps=1e-6, precision="fp32", stream=None):
        lib = load()
        R = L / 2.0 if R is None else float(R)
        h = ctypes.c_void_p()
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        _check(lib.ffb_plan(ctypes.byref(h), int(L), float(c), R, float(eps), prec, _stream(stream)),
               "ffb_plan")
        self._h = h
        info = (ctypes.c_int * 11)()
        _check(lib.ffb_plan_info(h, info), "ffb_plan_info")
        (self.L, self.k_max, self.P, self.n_xi, self.n_theta, self.N, self.w,
         self.precision, self.pmax, self.chunk, self.polar_variant) = list(info)
        self.c, self.R, self.eps = float(c), R, float(eps)
        pk = (ctypes.c_int * (self.k_max + 1))()
        off = (ctypes.c_int * (self.k_max + 1))()
        _check(lib.ffb_plan_sizes(h, pk, off), "ffb_plan_sizes")
        self.p = list(pk)
        self.offset = list(off)
        self.cov_total = sum(v * v for v in self.p)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ffb_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- host-side accessors ------------------------------------------------
    def tables(self):
        """float64 setup tables: (zeros[P], xi[n_xi], w[n_xi], B[P, n_xi])."""
        import numpy as np
        z = np.zeros(self.P)
        xi = np.zeros(self.n_xi)
        w = np.zeros(self.n_xi)
        B = np.zeros((self.P, self.n_xi))
        f = lambda a: a.ctypes.data_as(_pd)
        _check(load().ffb_plan_tables(self._h, f(z), f(xi), f(w), f(B)), "ffb_plan_tables")
        return z, xi, w, B

    def set_precision(self, precision):
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        _check(load().ffb_set_precision(self._h, prec), "ffb_set_precision")
        self.precision = prec

    def set_wait_budget(self, cycles=-1):
        """Bound of the tensor-core kernels' inter-role waits in clock cycles
        (tests of the timeout path); negative restores the default."""
        _check(load().ffb_set_wait_budget(self._h, int(cycles)), "ffb_set_wait_budget")

    KERNEL_CLASSES = ["rows_fft", "cols_fft", "interp_ring", "bessel", "covariance", "cov_aux", "jacobi",
                      "adj_bessel", "adj_ring_spread", "adj_cols", "adj_rows", "filter", "setup",
                      "grid_interp", "ring_fft", "adj_spread"]

    def profile(self, enable=True, stride=1):
        """Time every ``stride``-th launch of each kernel class (off if not enable)."""
        _check(load().ffb_profile(self._h, int(stride) if enable else 0), "ffb_profile")

    def profile_read(self):
        """{class: (total_ms, launches)} since profile(True); with a stride,
        total_ms is the timed launches' mean times the launch count."""
        ms = (ctypes.c_double * 16)()
        calls = (ctypes.c_int64 * 16)()
        _check(load().ffb_profile_read(self._h, ms, calls), "ffb_profile_read")
        return {name: (ms[i], int(calls[i])) for i, name in enumerate(self.KERNEL_CLASSES) if calls[i]}

    def launch_count(self):
        return int(load().ffb_launch_count(self._h))

    # -- compute (all asynchronous on the current stream unless noted) ------
    def polar(self, images, out=None, stream=None):
        n = images.shape[0]
        if out is None:
            out = torch.empty((n, self.n_xi, self.n_theta // 2, 2), device=images.device, dtype=torch.float32)
        _check(load().ffb_polar(self._h, _ptr(images, torch.float32, "images"), n,
                                _ptr(out, torch.float32, "out"), _stream(stream)), "ffb_polar")
        return out

    def expand(self, images, out=None, stream=None):
        """images float32 (n, L, L) -> coefficients float32 (n, P, 2)."""
        n = images.shape[0]
        if out is None:
            out = torch.empty((n, self.P, 2), device=images.device, dtype=torch.float32)
        _check(load().ffb_expand(self._h, _ptr(images, torch.float32, "images"), n,
                                 _ptr(out, torch.float32, "out"), _stream(stream)), "ffb_expand")
        return out

    def expand_adjoint(self, coef, out=None, stream=None):
        """coefficients float32 (n, P, 2) -> images float32 (n, L, L)."""
        n = coef.shape[0]
        if out is None:
            out = torch.empty((n, self.L, self.L), device=coef.device, dtype=torch.float32)
        _check(load().ffb_expand_adjoint(self._h, _ptr(coef, torch.float32, "coef"), n,
                                         _ptr(out, torch.float32, "out"), _stream(stream)),
               "ffb_expand_adjoint")
        return out

    def covariance(self, coef, reset=True, stream=None):
        n = coef.shape[0]
        _check(load().ffb_covariance(self._h, _ptr(coef, torch.float32, "coef"), n, int(bool(reset)),
                                     _stream(stream)), "ffb_covariance")

    def cov_get(self, device="cuda", stream=None):
        """Synchronising: (mean0 float64 (p_0,), packed C float64 (sum p_k^2,))."""
        mean = torch.empty(self.p[0], device=device, dtype=torch.float64)
        C = torch.empty(self.cov_total, device=device, dtype=torch.float64)
        _check(load().ffb_cov_get(self._h, _ptr(mean, torch.float64, "mean"), _ptr(C, torch.float64, "C"),
                                  _stream(stream)), "ffb_cov_get")
        return mean, C

    def expand_cov_host(self, images, reset=True, mean_out=None, C_out=None, stream=None):
        """Synchronising: host images float32 (n, L, L) (pinned for full copy
        bandwidth) -> expansion and covariance accumulation on the device ->
        (mean0 float64 (p_0,), packed C float64 (sum p_k^2,)) in host memory
        (ffb_expand_cov_host).  mean_out / C_out: optional host float64
        tensors to fill."""
        n = images.shape[0]
        mean = torch.empty(self.p[0], dtype=torch.float64) if mean_out is None else mean_out
        C = torch.empty(self.cov_total, dtype=torch.float64) if C_out is None else C_out
        if mean.numel() < self.p[0] or C.numel() < self.cov_total:
            raise ValueError("mean_out / C_out too small")
        _check(load().ffb_expand_cov_host(self._h, _hptr(images, torch.float32, "images"), n, int(bool(reset)),
                                          _hptr(mean, torch.float64, "mean_out"), _hptr(C, torch.float64, "C_out"),
                                          _stream(stream)), "ffb_expand_cov_host")
        return mean, C

    def state_len(self):
        return 1 + self.p[0] + self.cov_total

    def cov_export(self, stream=None):
        """Synchronising: float64 numpy state [n, mean0, packed C]."""
        import numpy as np
        st = np.zeros(self.state_len())
        _check(load().ffb_cov_export(self._h, st.ctypes.data_as(_pd), _stream(stream)), "ffb_cov_export")
        return st

    def cov_import(self, state, stream=None):
        import numpy as np
        st = np.ascontiguousarray(state, dtype=np.float64)
        _check(load().ffb_cov_import(self._h, st.ctypes.data_as(_pd), _stream(stream)), "ffb_cov_import")

    def eig(self, device="cuda", stream=None):
        """Synchronising: (evals float64 (P,), packed evecs float64 (sum p_k^2,))."""
        ev = torch.empty(self.P, device=device, dtype=torch.float64)
        U = torch.empty(self.cov_total, device=device, dtype=torch.float64)
        _check(load().ffb_eig(self._h, _ptr(ev, torch.float64, "evals"), _ptr(U, torch.float64, "evecs"),
                              _stream(stream)), "ffb_eig")
        return ev, U

    def svd(self, coef, device="cuda", stream=None):
        """Eigenpairs by the SVD route (ffb_svd): (evals [P], evecs packed)."""
        ev = torch.empty(self.P, dtype=torch.float64, device=device)
        U = torch.empty(self.cov_total, dtype=torch.float64, device=device)
        _check(load().ffb_svd(self._h, _ptr(coef, torch.float32, "coef"), coef.shape[0], _ptr(ev, torch.float64, "ev"),
                              _ptr(U, torch.float64, "U"), _stream(stream)), "ffb_svd")
        return ev, U

    def invariants(self, coef, pairs=(), triples=(), stream=None):
        """Rotation-invariant features (ffb_invariants): power [n, len(pairs)]
        and bispectrum [n, len(triples), 2]."""
        n = coef.shape[0]
        pw = torch.empty((n, len(pairs)), dtype=torch.float32, device=coef.device)
        bs = torch.empty((n, len(triples), 2), dtype=torch.float32, device=coef.device)
        hp = (ctypes.c_int * max(1, 2 * len(pairs)))(*[v for pr in pairs for v in pr])
        ht = (ctypes.c_int * max(1, 5 * len(triples)))(*[v for tr in triples for v in tr])
        _check(load().ffb_invariants(self._h, _ptr(coef, torch.float32, "coef"), n, len(pairs), hp,
                                     ctypes.c_void_p(pw.data_ptr()), len(triples), ht,
                                     ctypes.c_void_p(bs.data_ptr()), _stream(stream)), "ffb_invariants")
        return pw, bs

    def eig_blocks(self, C, stream=None):
        """Synchronising: Jacobi eigenpairs of caller-supplied packed blocks."""
        ev = torch.empty(self.P, device=C.device, dtype=torch.float64)
        U = torch.empty(self.cov_total, device=C.device, dtype=torch.float64)
        _check(load().ffb_eig_blocks(self._h, _ptr(C, torch.float64, "C"), _ptr(ev, torch.float64, "evals"),
                                     _ptr(U, torch.float64, "evecs"), _stream(stream)), "ffb_eig_blocks")
        return ev, U

    def radial_eigenfunctions(self, stream=None):
        """float64 (n_xi * P,) packed: block k at offset[k]*n_xi as (n_xi, p_k)."""
        out = torch.empty(self.n_xi * self.P, device="cuda", dtype=torch.float64)
        _check(load().ffb_radial_eigenfunctions(self._h, _ptr(out, torch.float64, "out"), _stream(stream)),
               "ffb_radial_eigenfunctions")
        return out

    def radial_block(self, packed, k):
        o, pk = self.offset[k], self.p[k]
        return packed[o * self.n_xi:(o + pk) * self.n_xi].view(self.n_xi, pk)

    def eigenimages(self, pairs, stream=None):
        """Complex128 (len(pairs), L, L) eigenimages of the (k, l) pairs."""
        ks = (ctypes.c_int * len(pairs))(*[int(k) for k, _ in pairs])
        ls = (ctypes.c_int * len(pairs))(*[int(l) for _, l in pairs])
        out = torch.empty((len(pairs), self.L, self.L, 2), device="cuda", dtype=torch.float64)
        _check(load().ffb_eigenimages(self._h, len(pairs), ks, ls, _ptr(out, torch.float64, "out"),
                                      _stream(stream)), "ffb_eigenimages")
        return torch.view_as_complex(out)

    def select(self, mode="topk", K=0, sigma2=0.0, n=0, stream=None):
        """Synchronising: gains h (numpy, P) of the selected components; stores
        the filter matrices in the plan."""
        import numpy as np
        m = DENOISE[mode] if isinstance(mode, str) else int(mode)
        h = np.zeros(self.P)
        _check(load().ffb_select(self._h, m, int(K), float(sigma2), int(n), h.ctypes.data_as(_pd),
                                 _stream(stream)), "ffb_select")
        return h

    def filter(self, coef, linear=False, weight=False, out=None, stream=None):
        n = coef.shape[0]
        if out is None:
            out = torch.empty_like(coef)
        flags = (1 if linear else 0) | (2 if weight else 0)
        _check(load().ffb_filter(self._h, _ptr(coef, torch.float32, "coef"), n, _ptr(out, torch.float32, "out"),
                                 flags, _stream(stream)), "ffb_filter")
        return out

    def weight(self, coef, out=None, stream=None):
        n = coef.shape[0]
        if out is None:
            out = torch.empty_like(coef)
        _check(load().ffb_weight(self._h, _ptr(coef, torch.float32, "coef"), n, _ptr(out, torch.float32, "out"),
                                 _stream(stream)), "ffb_weight")
        return out

    def synthesize(self, coef, out=None, stream=None):
        """Real images of the truncated expansion: adjoint(W a)."""
        return self.expand_adjoint(self.weight(coef, stream=stream), out=out, stream=stream)

    def denoise(self, images, mode="topk", K=0, sigma2=0.0, out=None, stream=None):
        n = images.shape[0]
        if out is None:
            out = torch.empty_like(images)
        m = DENOISE[mode] if isinstance(mode, str) else int(mode)
        _check(load().ffb_denoise(self._h, _ptr(images, torch.float32, "images"), n, m, int(K),
                                  float(sigma2), _ptr(out, torch.float32, "out"), _stream(stream)),
               "ffb_denoise")
        return out

    def sync(self, stream=None):
        _check(load().ffb_sync(self._h, _stream(stream)), "ffb_sync")

    def estimate_support(self, images, frac=0.999, sigma2=None, stream=None):
        """R, c and the noise variance of a stack (see ffb_estimate_support);
        returns a dict with the radial variance and radial power profiles."""
        import numpy as np
        n = images.shape[0]
        if tuple(images.shape[1:]) != (self.L, self.L):
            raise ValueError("images must be [n, L, L]")
        out = np.zeros(4)
        rv = np.zeros(self.L // 2)
        rp = np.zeros(self.n_xi)
        _check(load().ffb_estimate_support(self._h, _ptr(images, torch.float32, "images"), n, float(frac),
                                           -1.0 if sigma2 is None else float(sigma2),
                                           out.ctypes.data_as(_pd), rv.ctypes.data_as(_pd),
                                           rp.ctypes.data_as(_pd), _stream(stream)), "ffb_estimate_support")
        return {"R": out[0], "c": out[1], "sigma2": out[2], "c_index": int(out[3]),
                "radial_variance": rv, "radial_power": rp}

    # -- helpers for packed outputs ----------------------------------------
    def unpack_blocks(self, packed):
        """Packed (sum p_k^2,) -> list of (p_k, p_k) views."""
        out, o = [], 0
        for pk in self.p:
            out.append(packed[o:o + pk * pk].view(pk, pk))
            o += pk * pk
        return out


class Group:
    """Several stacks of uneven L and n through a1-a7 in one call (see the
    batching section of include/ffb.h).  ``plans`` are distinct Plans of one
    precision; they must outlive the group."""

    INFO = ("S", "precision", "per", "tile", "grid", "graphs", "replays", "eager", "launches", "candidates",
            "quad_per_sm", "quad_stages", "quad_candidates", "quad_rounds")

    def __init__(self, plans, stream=None):
        lib = load()
        self.plans = list(plans)
        hs = (_vp * len(self.plans))(*[p.handle.value for p in self.plans])
        self._h = _vp()
        _check(lib.ffb_group_create(ctypes.byref(self._h), len(self.plans), hs, _stream(stream)),
               "ffb_group_create")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ffb_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arrays(self, tensors, dtype, name, allow_none):
        ptrs = []
        for i, t in enumerate(tensors):
            if t is None and allow_none[i]:
                ptrs.append(None)
            else:
                ptrs.append(_ptr(t, dtype, "%s[%d]" % (name, i)).value)
        return (_vp * len(ptrs))(*ptrs)

    def expand_cov(self, images, coefs, reset=True, stream=None):
        """images[s]: float32 [n_s, L_s, L_s]; coefs[s]: float32 [n_s, P_s, 2]
        written by the call.  Returns coefs."""
        if len(images) != len(self.plans) or len(coefs) != len(self.plans):
            raise ValueError("one images and one coefficient tensor per stack")
        n = [0 if x is None else int(x.shape[0]) for x in images]
        for s, (p, x, c) in enumerate(zip(self.plans, images, coefs)):
            if n[s] and (tuple(x.shape[1:]) != (p.L, p.L) or c is None or tuple(c.shape) != (n[s], p.P, 2)):
                raise ValueError("stack %d: shapes do not match its plan" % s)
        zero = [v == 0 for v in n]
        _check(load().ffb_group_expand_cov(self._h, self._arrays(images, torch.float32, "images", zero),
                                           (ctypes.c_int64 * len(n))(*n),
                                           self._arrays(coefs, torch.float32, "coefs", zero), int(bool(reset)),
                                           _stream(stream)), "ffb_group_expand_cov")
        return coefs

    def covariance(self, coefs, reset=True, stream=None):
        n = [0 if c is None else int(c.shape[0]) for c in coefs]
        for s, (p, c) in enumerate(zip(self.plans, coefs)):
            if n[s] and tuple(c.shape[1:]) != (p.P, 2):
                raise ValueError("stack %d: coefficient shape does not match its plan" % s)
        zero = [v == 0 for v in n]
        _check(load().ffb_group_covariance(self._h, self._arrays(coefs, torch.float32, "coefs", zero),
                                           (ctypes.c_int64 * len(n))(*n), int(bool(reset)), _stream(stream)),
               "ffb_group_covariance")

    def sync(self, stream=None):
        _check(load().ffb_group_sync(self._h, _stream(stream)), "ffb_group_sync")

    def info(self):
        out = (ctypes.c_int64 * 14)()
        _check(load().ffb_group_info(self._h, out), "ffb_group_info")
        return dict(zip(self.INFO, list(out)))

    def tuning(self):
        m = 32
        per, tile, grid = (ctypes.c_int * m)(), (ctypes.c_int * m)(), (ctypes.c_int * m)()
        ms = (ctypes.c_float * m)()
        k = load().ffb_group_tuning(self._h, m, per, tile, grid, ms)
        if k < 0:
            raise FFBError(k, "ffb_group_tuning")
        return [{"per": per[i], "tile": tile[i], "grid": grid[i], "ms": ms[i]} for i in range(k)]

    def quad_tuning(self):
        """Timed launch shapes of the grouped quadrature: CTAs per SM, stages, ms."""
        m = 8
        per, st = (ctypes.c_int * m)(), (ctypes.c_int * m)()
        ms = (ctypes.c_float * m)()
        k = load().ffb_group_quad_tuning(self._h, m, per, st, ms)
        if k < 0:
            raise FFBError(k, "ffb_group_quad_tuning")
        return [{"per_sm": per[i], "stages": st[i], "ms": ms[i]} for i in range(k)]
