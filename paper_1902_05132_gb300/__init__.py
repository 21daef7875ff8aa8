"""GB300 layered-media Helmholtz FMM: thin ctypes binding of libfmmlayered.so.

Argument marshalling only: every step of the evaluation runs in the library's
CUDA kernels.  The library is built in-tree by ``_build.build()``; importing
this package does not build it, and every call fails loudly if it is missing.

Tensors: positions float64 [N, 3] (row-major), charges complex128 [N],
results complex128 [N], all on the CUDA device the solver was created on
(``eval``/``direct``), or numpy arrays in host memory (``eval_host``).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfmmlayered.so")

FMM_PLAIN_FP64 = 0
FMM_NORM_PAPER = 1
FMM_MIXED = 2
FMM_SURROGATE = 4
FMM_TREE_COUNTS = 8
FMM_TABLES = 16
SURR_CELLS = 512          # cells of the surrogate's held-out check (8 x 8 x 8)
FMM_TEST_STALL_TC = 1 << 30

ERRORS = {0: "ok", -1: "invalid argument", -2: "point on an interface", -3: "non-finite input",
          -4: "CUDA error", -5: "out of device memory", -6: "timeout", -7: "unsupported"}


class FmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("n_components", ctypes.c_int), ("n_boxes", ctypes.c_int), ("max_level", ctypes.c_int),
                ("n_v_pairs", ctypes.c_long), ("n_u_pairs", ctypes.c_long), ("n_quad_near", ctypes.c_int),
                ("n_quad_total", ctypes.c_int), ("ms_setup", ctypes.c_double), ("ms_tree", ctypes.c_double),
                ("ms_operators", ctypes.c_double), ("ms_eval", ctypes.c_double),
                ("gpu_ms_tree", ctypes.c_double), ("gpu_ms_operators", ctypes.c_double),
                ("gpu_ms_upward", ctypes.c_double), ("gpu_ms_m2l", ctypes.c_double),
                ("gpu_ms_l2p", ctypes.c_double), ("gpu_ms_near_free", ctypes.c_double),
                ("gpu_ms_near_reac", ctypes.c_double), ("gpu_ms_sum", ctypes.c_double),
                ("gpu_ms_total", ctypes.c_double), ("n_free_pairs", ctypes.c_long),
                ("n_reac_pairs", ctypes.c_long), ("n_reac_nodes", ctypes.c_long),
                ("n_reac_tail_nodes", ctypes.c_long), ("n_reac_classes", ctypes.c_long),
                ("n_free_ops", ctypes.c_long), ("n_reac_T_nodes", ctypes.c_long),
                ("n_v_pairs_reac", ctypes.c_long), ("n_launches", ctypes.c_long),
                ("gpu_ms_m2l_gemm", ctypes.c_double), ("m2l_gemm_flops", ctypes.c_double),
                ("m2l_tensor_flops", ctypes.c_double), ("m2l_tc_bytes", ctypes.c_double),
                ("n_reac_surr_pairs", ctypes.c_long), ("reac_near_rho_max", ctypes.c_double),
                ("reac_near_z_min", ctypes.c_double), ("reac_near_z_max", ctypes.c_double),
                ("ms_tables", ctypes.c_double), ("table_bytes", ctypes.c_double),
                ("n_reac_table_classes", ctypes.c_long), ("n_reac_table_pairs", ctypes.c_long),
                ("tune_zrot_kc", ctypes.c_int), ("tune_zrot_threads", ctypes.c_int),
                ("tune_zrot_candidates", ctypes.c_int), ("tune_zrot_ms", ctypes.c_double),
                ("tune_zrot_rule_ms", ctypes.c_double)]


EXPORTED = ["fmm_layered_create", "fmm_layered_destroy", "fmm_layered_last_error", "fmm_layered_eval",
            "fmm_layered_eval_host", "fmm_layered_direct", "fmm_layered_stats",
            "fmm_layered_num_components", "fmm_layered_component_info", "fmm_layered_tree_export",
            "fmm_layered_measure_fp64_peak", "fmm_layered_direct_noalloc", "fmm_layered_eval_batched",
            "fmm_layered_surrogate_train", "fmm_layered_surrogate_report", "fmm_layered_surrogate_set_bound",
            "fmm_layered_surrogate_grad", "fmm_layered_set_components", "fmm_layered_component_work",
            "fmm_layered_add_components", "fmm_layered_table_operator", "fmm_layered_share_workspace"]

_lib = None


def lib():
    """Load libfmmlayered.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1902_05132_gb300._build.build()")
    L = ctypes.CDLL(LIB_PATH)
    d, i, l, v, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_void_p, ctypes.c_uint
    L.fmm_layered_create.argtypes = [i, d, d, d, i, i, u, ctypes.POINTER(ctypes.c_void_p)]
    L.fmm_layered_create.restype = i
    L.fmm_layered_destroy.argtypes = [v]
    L.fmm_layered_destroy.restype = None
    L.fmm_layered_last_error.argtypes = [v]
    L.fmm_layered_last_error.restype = ctypes.c_char_p
    for name in ("fmm_layered_eval", "fmm_layered_eval_host", "fmm_layered_direct",
                 "fmm_layered_direct_noalloc"):
        f = getattr(L, name)
        f.argtypes = [v, l, d, d, l, d, d, v]
        f.restype = i
    L.fmm_layered_eval_batched.argtypes = [i, d, d, d, d, d, d, d, v]
    L.fmm_layered_eval_batched.restype = i
    L.fmm_layered_surrogate_train.argtypes = [v, ctypes.c_double, ctypes.c_double, ctypes.c_double, l, i,
                                              ctypes.c_double, ctypes.c_ulonglong, v]
    L.fmm_layered_surrogate_train.restype = i
    L.fmm_layered_surrogate_set_bound.argtypes = [v, ctypes.c_double]
    L.fmm_layered_surrogate_set_bound.restype = i
    L.fmm_layered_surrogate_report.argtypes = [v, d, d]
    L.fmm_layered_surrogate_report.restype = i
    L.fmm_layered_surrogate_grad.argtypes = [d, d, d, d]
    L.fmm_layered_surrogate_grad.restype = i
    L.fmm_layered_set_components.argtypes = [v, i, i]
    L.fmm_layered_set_components.restype = i
    L.fmm_layered_component_work.argtypes = [v, d, i]
    L.fmm_layered_component_work.restype = i
    L.fmm_layered_add_components.argtypes = [v, d, v]
    L.fmm_layered_add_components.restype = i
    L.fmm_layered_stats.argtypes = [v, ctypes.POINTER(Stats)]
    L.fmm_layered_stats.restype = i
    L.fmm_layered_num_components.argtypes = [v]
    L.fmm_layered_num_components.restype = i
    L.fmm_layered_component_info.argtypes = [v, i, d, d]
    L.fmm_layered_component_info.restype = i
    L.fmm_layered_tree_export.argtypes = [v, i] + [d] * 14
    L.fmm_layered_tree_export.restype = i
    L.fmm_layered_measure_fp64_peak.argtypes = [d]
    L.fmm_layered_measure_fp64_peak.restype = i
    L.fmm_layered_table_operator.argtypes = [v, i, i, i, i, ctypes.c_double, i, i, i, d]
    L.fmm_layered_table_operator.restype = i
    L.fmm_layered_share_workspace.argtypes = [v, v]
    L.fmm_layered_share_workspace.restype = i
    _lib = L
    return L


def eval_batched(solvers, problems, outs=None, stream=None):
    """Evaluate independent problems concurrently (fmm_layered_eval_batched).

    solvers: distinct LayeredFMM handles; problems: (src, q, tgt) device
    tensors per handle.  Returns the list of potentials."""
    import torch
    n = len(solvers)
    if len(problems) != n or len({id(s) for s in solvers}) != n:
        raise ValueError("one distinct solver per problem")
    args = [LayeredFMM._dev_args(*pr) for pr in problems]
    if outs is None:
        outs = [torch.empty(t.shape[0], dtype=torch.complex128, device=t.device) for _, _, t in args]
    outr = [torch.view_as_real(o) for o in outs]
    P = ctypes.c_void_p * n
    Lg = ctypes.c_long * n
    hs = P(*[s.h for s in solvers])
    ns = Lg(*[a[0].shape[0] for a in args])
    nt = Lg(*[a[2].shape[0] for a in args])
    src = P(*[_ptr(a[0]) for a in args])
    q = P(*[_ptr(a[1]) for a in args])
    tgt = P(*[_ptr(a[2]) for a in args])
    out = P(*[_ptr(o) for o in outr])
    if stream is None:
        stream = torch.cuda.current_stream(args[0][2].device if n else None)
    rc = lib().fmm_layered_eval_batched(n, ctypes.cast(hs, ctypes.c_void_p), ctypes.cast(ns, ctypes.c_void_p),
                                        ctypes.cast(src, ctypes.c_void_p), ctypes.cast(q, ctypes.c_void_p),
                                        ctypes.cast(nt, ctypes.c_void_p), ctypes.cast(tgt, ctypes.c_void_p),
                                        ctypes.cast(out, ctypes.c_void_p), ctypes.c_void_p(stream.cuda_stream))
    if rc != 0:
        msgs = [lib().fmm_layered_last_error(s.h).decode() for s in solvers]
        raise FmmError(rc, "; ".join(f"problem {i}: {m}" for i, m in enumerate(msgs) if m) or "invalid argument")
    return outs


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


class LayeredFMM:
    """Solver for one layered medium (Sec. 3.1): wave numbers k (top to bottom),
    interfaces d (descending), material coefficients eps, order p, leaf size.
    mixed=True runs the M2L translations on the tensor cores (FP16 hi/lo
    operands, FP32 accumulation); every other stage stays FP64.
    tree_counts=True refines reaction trees by the point counts alone
    (FMM_TREE_COUNTS), so reaction components get near-field pairs.
    tables=True tabulates the reaction M2L integrals at create (FMM_TABLES)
    and interpolates the reaction operators of every geometry from them."""

    def __init__(self, k, d=(), eps=None, p=8, leaf=64, paper_norm=False, mixed=False, surrogate=False,
                 tree_counts=False, tables=False, extra_flags=0):
        L = lib()
        self.k = np.ascontiguousarray(k, dtype=np.float64)
        self.d = np.ascontiguousarray(d, dtype=np.float64)
        self.eps = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
        self.p, self.leaf = int(p), int(leaf)
        h = ctypes.c_void_p()
        rc = L.fmm_layered_create(len(self.k), _ptr(self.k), _ptr(self.d) if len(self.d) else None,
                                  _ptr(self.eps), self.p, self.leaf,
                                  (FMM_NORM_PAPER if paper_norm else FMM_PLAIN_FP64) | (FMM_MIXED if mixed else 0)
                                  | (FMM_SURROGATE if surrogate else 0) | (FMM_TREE_COUNTS if tree_counts else 0)
                                  | (FMM_TABLES if tables else 0) | int(extra_flags),
                                  ctypes.byref(h))
        if rc != 0:
            raise FmmError(rc, L.fmm_layered_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().fmm_layered_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise FmmError(rc, lib().fmm_layered_last_error(self.h).decode())

    @staticmethod
    def _dev_args(src, q, tgt):
        import torch
        src = src.contiguous()
        tgt = tgt.contiguous()
        qr = torch.view_as_real(q.contiguous()).contiguous()
        return src, qr, tgt

    def _call_dev(self, fn, src, q, tgt, out, stream):
        import torch
        src, qr, tgt = self._dev_args(src, q, tgt)
        if out is None:
            out = torch.empty(tgt.shape[0], dtype=torch.complex128, device=tgt.device)
        outr = torch.view_as_real(out)
        if stream is None:
            stream = torch.cuda.current_stream(tgt.device)
        self._check(fn(self.h, src.shape[0], _ptr(src), _ptr(qr), tgt.shape[0], _ptr(tgt), _ptr(outr),
                       ctypes.c_void_p(stream.cuda_stream)))
        return out

    def eval(self, src, q, tgt, out=None, stream=None):
        """FMM potentials at tgt (device tensors)."""
        return self._call_dev(lib().fmm_layered_eval, src, q, tgt, out, stream)

    def direct(self, src, q, tgt, out=None, stream=None):
        """All-pairs direct sum on the GPU (device tensors)."""
        return self._call_dev(lib().fmm_layered_direct, src, q, tgt, out, stream)

    def direct_noalloc(self, src, q, tgt, out=None, stream=None):
        """Direct sum that allocates no device memory (fixed library scratch;
        see fmm_layered_direct_noalloc).  Pass ``out`` to avoid the one torch
        allocation this wrapper would otherwise make for the result."""
        return self._call_dev(lib().fmm_layered_direct_noalloc, src, q, tgt, out, stream)

    def eval_host(self, src, q, tgt, stream=None):
        """FMM with host (numpy) buffers: copies in, evaluates, copies back."""
        src = np.ascontiguousarray(src, dtype=np.float64)
        tgt = np.ascontiguousarray(tgt, dtype=np.float64)
        qr = np.ascontiguousarray(np.asarray(q, dtype=np.complex128)).view(np.float64)
        out = np.empty(2 * len(tgt), dtype=np.float64)
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self._check(lib().fmm_layered_eval_host(self.h, len(src), _ptr(src), _ptr(qr), len(tgt), _ptr(tgt),
                                                _ptr(out), st))
        return out.view(np.complex128)

    def train_surrogate(self, rho_max, z_min, z_max, samples=16384, steps=2000, bound=1e-5, seed=0, stream=None):
        """Train the learned surrogate of the reaction components
        (fmm_layered_surrogate_train); returns the per-cell report."""
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        self._check(lib().fmm_layered_surrogate_train(self.h, float(rho_max), float(z_min), float(z_max),
                                                      int(samples), int(steps), float(bound),
                                                      ctypes.c_ulonglong(seed), st))
        return self.surrogate_report()

    def surrogate_set_bound(self, bound):
        """Use the surrogate only in cells whose held-out error is within `bound`."""
        self._check(lib().fmm_layered_surrogate_set_bound(self.h, float(bound)))
        return self.surrogate_report()

    def surrogate_report(self):
        """(cell_err, cell_ok), shape [4 L1^2, 512]; slot ((l*L1 + l')*2 + a)*2 + b,
        cell (c_rho*8 + c_zt)*8 + c_zs."""
        n = 4 * len(self.k) ** 2 * SURR_CELLS
        err = np.zeros(n, dtype=np.float64)
        ok = np.zeros(n, dtype=np.uint8)
        self._check(lib().fmm_layered_surrogate_report(self.h, _ptr(err), _ptr(ok)))
        return err.reshape(-1, SURR_CELLS), ok.reshape(-1, SURR_CELLS).astype(bool)

    def set_components(self, first=0, count=-1):
        """Evaluate only components [first, first + count) (count < 0: all)."""
        self._check(lib().fmm_layered_set_components(self.h, int(first), int(count)))

    def component_work(self):
        """Work estimate of each component of the last evaluation."""
        n = lib().fmm_layered_num_components(self.h)
        w = np.zeros(max(n, 1), dtype=np.float64)
        rc = lib().fmm_layered_component_work(self.h, _ptr(w), len(w))
        if rc < 0:
            self._check(rc)
        return w[:rc]

    def add_components(self, out, stream=None):
        """out (complex128 device tensor) += the last evaluation's component
        potentials, one component after the other in their order."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(out.device)
        self._check(lib().fmm_layered_add_components(self.h, _ptr(torch.view_as_real(out)),
                                                     ctypes.c_void_p(stream.cuda_stream)))
        return out

    def share_workspace(self, owner):
        """Use the device workspace of another handle (fmm_layered_share_workspace);
        the two must then not be evaluated at the same time."""
        self._check(lib().fmm_layered_share_workspace(self.h, owner.h))

    def table_operator(self, l, lp, a, b, w, jt, js, r):
        """Radial reaction M2L operator of one class interpolated from the
        tables (fmm_layered_table_operator): complex [(p+1)^2][(p+1)^2], rows
        the output coefficients (n, m), columns the input ones."""
        P = (self.p + 1) ** 2
        out = np.zeros((P, P), dtype=np.complex128)
        self._check(lib().fmm_layered_table_operator(self.h, int(l), int(lp), int(a), int(b), float(w), int(jt),
                                                     int(js), int(r), _ptr(out.view(np.float64))))
        return out

    def stats(self):
        s = Stats()
        self._check(lib().fmm_layered_stats(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def trees(self):
        """Trees and lists of the last evaluation, one dict per component."""
        L = lib()
        out = []
        for c in range(L.fmm_layered_num_components(self.h)):
            info = np.zeros(10, dtype=np.int64)
            root = np.zeros(4, dtype=np.float64)
            self._check(L.fmm_layered_component_info(self.h, c, _ptr(info), _ptr(root)))
            kind, l, lp, a, b, ns, nt, nb, nlev, _ = (int(x) for x in info)
            arr = {name: np.zeros(nb, dtype=np.int32) for name in
                   ("level", "src_begin", "src_end", "tgt_begin", "tgt_end", "parent")}
            prefix = np.zeros(nb, dtype=np.int64)
            sperm = np.zeros(max(ns, 1), dtype=np.int32)
            tperm = np.zeros(max(nt, 1), dtype=np.int32)
            off = np.zeros(4 * (nb + 1), dtype=np.int32)
            self._check(L.fmm_layered_tree_export(self.h, c, _ptr(arr["level"]), _ptr(prefix), _ptr(arr["src_begin"]),
                                                  _ptr(arr["src_end"]), _ptr(arr["tgt_begin"]), _ptr(arr["tgt_end"]),
                                                  _ptr(arr["parent"]), _ptr(sperm), _ptr(tperm), _ptr(off),
                                                  None, None, None, None))
            off = off.reshape(4, nb + 1)
            idx = [np.zeros(max(int(off[k, nb]), 1), dtype=np.int32) for k in range(4)]
            self._check(L.fmm_layered_tree_export(self.h, c, None, None, None, None, None, None, None, None, None,
                                                  _ptr(off), *(_ptr(x) for x in idx)))
            lists = {}
            for k, name in enumerate("VUWX"):
                lists[name] = {bx: idx[k][off[k, bx]:off[k, bx + 1]].tolist()
                               for bx in range(nb) if off[k, bx + 1] > off[k, bx]}
            out.append(dict(kind=kind, l=l, lp=lp, a=a, b=b, ns=ns, nt=nt, root=root, prefix=prefix.view(np.uint64),
                            sperm=sperm[:ns], tperm=tperm[:nt], lists=lists, **arr))
        return out


SURR_NPARAM = 8706
SURR_BATCH = 1024


def surrogate_grad(params, x, y):
    """Gradient of the surrogate's training loss over one minibatch by the
    library's training kernels (fmm_layered_surrogate_grad): params float32
    [8706], x float32 [1024, 3], y float32 [1024, 2] (host arrays)."""
    params = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    if params.shape != (SURR_NPARAM,) or x.shape != (SURR_BATCH, 3) or y.shape != (SURR_BATCH, 2):
        raise ValueError("params [8706], x [1024, 3], y [1024, 2]")
    g = np.zeros(SURR_NPARAM, dtype=np.float32)
    rc = lib().fmm_layered_surrogate_grad(_ptr(params), _ptr(x), _ptr(y), _ptr(g))
    if rc != 0:
        raise FmmError(rc, "surrogate gradient failed")
    return g


def measure_fp64_peak():
    """Dependent-FMA FP64 throughput of the current device, GFLOP/s."""
    v = ctypes.c_double()
    rc = lib().fmm_layered_measure_fp64_peak(ctypes.byref(v))
    if rc != 0:
        raise FmmError(rc, "peak measurement failed")
    return v.value
