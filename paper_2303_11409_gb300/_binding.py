"""ctypes binding of the C ABI in include/mps_gb300.h.

Argument marshalling only: every step of the two-site update runs in the CUDA
library.  The library must have been built (python -m paper_2303_11409_gb300.build);
importing this module fails loudly otherwise.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmps_gb300.so")

MPS_OK, MPS_EINVAL, MPS_ECHARGE, MPS_ENOMEM, MPS_ENOCONV, MPS_ECUDA, MPS_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
MPS_FP64, MPS_TF32, MPS_BF16X3 = 0, 1, 2
MPS_MAX_D = 8
MPS_NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024
KERNEL_KINDS = ("theta", "svd", "select", "lambda", "scatter", "gemm", "expect", "amplitude", "sample", "tcgemm",
                "shadow")
STATUS_NAMES = {0: "MPS_OK", -1: "MPS_EINVAL", -2: "MPS_ECHARGE", -3: "MPS_ENOMEM", -4: "MPS_ENOCONV",
                -5: "MPS_ECUDA", -6: "MPS_ETIMEOUT"}


class MPSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class JacobiNotConverged(UserWarning):
    pass


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"CUDA library {LIB_PATH} is not built; run `python -m paper_2303_11409_gb300.build` "
            "(there is no CPU fallback)")
    return ctypes.CDLL(LIB_PATH)


lib = _load()

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_intp = ctypes.POINTER(ctypes.c_int)
_dblp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_h = ctypes.c_void_p

_SIGS = {
    "mps_create": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_int, ctypes.c_int, _i32p, ctypes.c_int,
                                  ctypes.c_int, _vp]),
    "mps_create_segment": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_int, ctypes.c_int, _i32p, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "mps_destroy": (ctypes.c_int, [_h]),
    "mps_last_error": (ctypes.c_char_p, [_h]),
    "mps_info": (ctypes.c_int, [_h, _intp, _intp, _intp, _intp, _intp]),
    "mps_apply_gate2": (ctypes.c_int, [_h, ctypes.c_int, _dblp, ctypes.c_int, ctypes.c_double, _dblp]),
    "mps_apply_layer": (ctypes.c_int, [_h, ctypes.c_int, _intp, ctypes.POINTER(_dblp), ctypes.c_int,
                                       ctypes.c_double, _dblp]),
    "mps_apply_gate2_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_h), _intp, ctypes.POINTER(_dblp),
                                             _intp, _dblp, _dblp, _intp]),
    "mps_exec_create": (ctypes.c_int, [ctypes.POINTER(_h), _vp]),
    "mps_exec_destroy": (ctypes.c_int, [_h]),
    "mps_exec_apply": (ctypes.c_int, [_h, ctypes.c_int, ctypes.POINTER(_h), _intp, ctypes.POINTER(_dblp), _intp,
                                      _dblp, _dblp, _intp]),
    "mps_footprint_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p, _i64p]),
    "mps_expect": (ctypes.c_int, [_h, ctypes.c_int, _dblp, _dblp]),
    "mps_amplitude": (ctypes.c_int, [_h, _i32p, _dblp]),
    "mps_amplitude_batch": (ctypes.c_int, [_h, ctypes.c_int, _i32p, _dblp]),
    "mps_sample": (ctypes.c_int, [_h, ctypes.c_int, _dblp, _i32p, _dblp]),
    "mps_bond_spectrum": (ctypes.c_int, [_h, ctypes.c_int, _i32p, _i32p, _dblp, ctypes.c_int, _intp]),
    "mps_bond_entropy": (ctypes.c_int, [_h, ctypes.c_int, _dblp]),
    "mps_save": (ctypes.c_int, [_h, ctypes.c_char_p]),
    "mps_load": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_char_p, _vp]),
    "mps_get_site": (ctypes.c_int, [_h, ctypes.c_int, _i32p, _i32p, ctypes.c_int, _dblp, ctypes.c_int64,
                                    _intp, _i64p]),
    "mps_set_bond": (ctypes.c_int, [_h, ctypes.c_int, ctypes.c_int, _i32p, _i32p, _dblp]),
    "mps_set_site": (ctypes.c_int, [_h, ctypes.c_int, ctypes.c_int, _i32p, _i32p, _dblp]),
    "mps_last_update_stats": (ctypes.c_int, [_h, _intp, _intp, _intp, _intp, _dblp, _dblp]),
    "mps_deflation_stats": (ctypes.c_int, [_h, _i64p, _i64p]),
    "mps_plan_sectors": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i32p, _i32p, ctypes.c_int, _i32p, _i32p,
                                        ctypes.c_int, _i32p, _i32p, _i32p, ctypes.c_int, _intp, _i32p,
                                        ctypes.c_int, _intp]),
    "mps_plan_sectors_rule": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _i32p,
                                             ctypes.c_int, _i32p, _i32p, ctypes.c_int, _i32p, _i32p,
                                             ctypes.c_int, _i32p, _i32p, _i32p, ctypes.c_int, _intp, _i32p,
                                             ctypes.c_int, _intp, _i32p, ctypes.c_int, _intp]),
    "mps_gate_layout": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _i32p, ctypes.c_int,
                                       _intp, _i64p]),
    "mps_last_batch_sweeps": (ctypes.c_int, [_h, _intp, _i64p, _intp]),
    "mps_set_profiling": (ctypes.c_int, [_h, ctypes.c_int]),
    "mps_kernel_stats": (ctypes.c_int, [_h, ctypes.c_int, _i64p, _dblp, _dblp, _dblp]),
    "mps_reset_kernel_stats": (ctypes.c_int, [_h]),
    "mps_launch_count": (ctypes.c_int64, []),
    "mps_svd_work_bytes": (ctypes.c_int64, [ctypes.c_int, _intp, _intp]),
    "mps_fp64_peak_probe": (ctypes.c_int, [_dblp, _vp]),
    "mps_zgemm_tc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                    ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int64, _vp]),
    "mps_svd_sectors_noalloc": (ctypes.c_int, [ctypes.c_int, _intp, _intp, _vp, _i64p, _vp, _i64p, _vp, _i64p,
                                               _vp, _i64p, _vp, _vp]),
    "mps_svd_sectors": (ctypes.c_int, [ctypes.c_int, _intp, _intp, _vp, _i64p, _vp, _i64p, _vp, _i64p, _vp,
                                       _i64p, _vp, _vp, ctypes.c_int64, _vp]),
    "mps_set_graphs": (ctypes.c_int, [_h, ctypes.c_int]),
    "mps_set_sweep_limit": (ctypes.c_int, [_h, ctypes.c_int]),
    "mps_tc_inject_stall": (ctypes.c_int, [ctypes.c_int]),
    "mps_graph_stats": (ctypes.c_int, [_h, _i64p, _i64p, _i64p]),
    "mps_set_autotune": (ctypes.c_int, [_h, ctypes.c_int]),
    "mps_autotune_stats": (ctypes.c_int, [_i64p, _i64p, _i64p]),
    "mps_autotune_table": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int, _intp]),
    "mps_autotune_clear": (ctypes.c_int, []),
    "mps_autotune_min_flops": (ctypes.c_int, [ctypes.c_double]),
    "mps_autotune_freeze": (ctypes.c_int, [ctypes.c_int]),
    "mps_autotune_force": (ctypes.c_int, [ctypes.c_int]),
    "mps_set_chi_deflation": (ctypes.c_int, [_h, ctypes.c_double]),
    "mps_create_zn": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_int, ctypes.c_int, _i32p, ctypes.c_int,
                                     ctypes.c_int, _vp]),
    "mps_create_cyclic": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p,
                                         ctypes.c_int, ctypes.c_int, _vp]),
    "mps_zgemm_tc_work_bytes": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mps_svd_mixed_min_k": (ctypes.c_int, [ctypes.c_int]),
    "mps_svd_mixed_sweeps": (ctypes.c_int, [ctypes.c_int]),
    "mps_dmrg": (ctypes.c_int, [_h, ctypes.POINTER(_dblp), ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                ctypes.c_double, _dblp, ctypes.c_int, _intp]),
    "mps_dmrg_stats": (ctypes.c_int, [_h, ctypes.c_int, _i64p, _dblp, _dblp]),
    "mps_dmrg_counts": (ctypes.c_int, [_h, _i64p, _i64p]),
    "mps_create_multi": (ctypes.c_int, [ctypes.POINTER(_h), ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _i32p,
                                        ctypes.c_int, ctypes.c_int, _vp]),
    "mps_charge_radix": (ctypes.c_int, [_h, _intp, _i32p]),
    "mps_charge_rule": (ctypes.c_int, [_h, _intp, _intp, _i32p]),
    "mps_svd_cluster_min_k": (ctypes.c_int, [ctypes.c_int]),
    "mps_tdvp": (ctypes.c_int, [_h, ctypes.POINTER(_dblp), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                ctypes.c_double, ctypes.c_int, ctypes.c_double, _dblp, ctypes.c_int, _intp]),
}
DMRG_KINDS = ("heff", "env", "lanczos", "svd", "other")
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _c128_flat(blocks) -> np.ndarray:
    if isinstance(blocks, np.ndarray) and blocks.ndim == 1:
        flat = blocks
    else:
        flat = np.concatenate([np.asarray(b, dtype=np.complex128).reshape(-1) for b in blocks])
    return np.ascontiguousarray(flat, dtype=np.complex128)


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch is optional plumbing
        pass
    return None


def gate_length(d: int) -> int:
    """Complex numbers in one flattened gate: sum over n of s_n^2."""
    tot = 0
    for n in range(2 * d - 1):
        s = min(d - 1, n) - max(0, n - d + 1) + 1
        tot += s * s
    return tot


def multi_pair_blocks(charges):
    """Two-site gate layout of a several-U(1) handle: the totals q_i + q_j (tuples) ascending,
    each with its pairs (i, j), i ascending."""
    tot = {}
    for i, a in enumerate(charges):
        for j, b in enumerate(charges):
            tot.setdefault(tuple(x + y for x, y in zip(a, b)), []).append((i, j))
    return {Q: sorted(tot[Q]) for Q in sorted(tot)}


def cyclic_pair_blocks(n: int, d: int):
    """Two-site gate layout of a Z_n handle with local dimension d <= n: the residues q = (i + j)
    mod n that some pair reaches, ascending, each with its pairs (i, (q - i) mod n), i ascending."""
    out = {}
    for q in range(n):
        pairs = [(i, (q - i) % n) for i in range(d) if (q - i) % n < d]
        if pairs:
            out[q] = pairs
    return out


class MPS:
    """A U(1)-symmetric MPS living on the GPU (one handle of the C library); zn = n >= d makes it
    Z_n-symmetric instead (mps_create_zn for d = n, mps_create_cyclic for d < n); charges = [q_0, ..., q_{d-1}] (tuples, ascending)
    gives physical index i the several-U(1) charge q_i (mps_create_multi): bond charges and
    gate blocks are then keyed by tuples."""

    charges = None          # several-U(1) charge vectors (None: a single U(1) or Z_n charge)

    def __init__(self, d: int, occupations, chi_max: int, precision: int = MPS_FP64, stream=None, zn: int = 0,
                 charges=None):
        occ = _i32(occupations)
        self.L, self.d, self.chi_max = len(occ), int(d), int(chi_max)
        self.zn = int(zn)
        self.charges = [tuple(int(v) for v in q) for q in charges] if charges is not None else None
        self.stream = _default_stream() if stream is None else stream
        h = _h()
        if self.charges is not None:
            nc = len(self.charges[0])
            qa = _i32(np.asarray(self.charges, dtype=np.int32).reshape(-1))
            rc = lib.mps_create_multi(ctypes.byref(h), self.L, self.d, nc, _ptr(qa, _i32p), _ptr(occ, _i32p),
                                      precision, self.chi_max, self.stream)
            if rc != MPS_OK:
                raise MPSError(rc, "mps_create_multi failed")
            self._h = h
            self._set_multi_keys()
            self.N = tuple(sum(self.charges[i][k] for i in occ) for k in range(nc))
            return
        if self.zn:
            if self.zn < self.d:
                raise ValueError("a Z_n handle has d <= n")
            if self.zn == self.d:
                rc = lib.mps_create_zn(ctypes.byref(h), self.L, self.zn, _ptr(occ, _i32p), precision,
                                       self.chi_max, self.stream)
            else:
                rc = lib.mps_create_cyclic(ctypes.byref(h), self.L, self.d, self.zn, _ptr(occ, _i32p), precision,
                                           self.chi_max, self.stream)
        else:
            rc = lib.mps_create(ctypes.byref(h), self.L, self.d, _ptr(occ, _i32p), precision, self.chi_max,
                                self.stream)
        if rc != MPS_OK:
            raise MPSError(rc, "mps_create failed")
        self._h = h
        self.N = int(occ.sum()) % self.zn if self.zn else int(occ.sum())

    # -- several-U(1) charge keys -------------------------------------------------
    def _set_multi_keys(self):
        """The encoding weights, radices and gate layout of a several-U(1) handle."""
        nc = len(self.charges[0])
        ncomp = ctypes.c_int(0)
        rad = np.zeros(4, np.int32)
        lib.mps_charge_radix(self._h, ctypes.byref(ncomp), _ptr(rad, _i32p))
        w, self._weights = 1, [0] * nc
        for k in range(nc - 1, -1, -1):
            self._weights[k] = w
            w *= int(rad[k])
        self._radix = [int(x) for x in rad[:nc]]
        self._pairs = multi_pair_blocks(self.charges)

    def _enc(self, c):
        return int(sum(x * w for x, w in zip(c, self._weights))) if self.charges is not None else int(c)

    def _dec(self, v):
        if self.charges is None:
            return int(v)
        out = []
        for w in self._weights:
            out.append(int(v) // w)
            v = int(v) - out[-1] * w
        return tuple(out)

    def _gate_flat(self, gate):
        if self.charges is not None and isinstance(gate, dict):
            return _c128_flat([gate[Q] for Q in self._pairs])
        return _c128_flat(gate)

    def gate_length(self) -> int:
        """Complex numbers in one flattened gate of this handle's charge rule."""
        if self.charges is not None:
            return sum(len(p) ** 2 for p in self._pairs.values())
        if getattr(self, "zn", 0):
            return sum(len(p) ** 2 for p in cyclic_pair_blocks(self.zn, self.d).values())
        return gate_length(self.d)

    # -- checkpoint -------------------------------------------------------------
    def save(self, path) -> None:
        """Write the state to `path` (mps_save)."""
        self._check(lib.mps_save(self._h, os.fsencode(path)), "mps_save")

    @classmethod
    def load(cls, path, stream=None) -> "MPS":
        """A new handle holding the state saved at `path` (mps_load)."""
        obj = cls.__new__(cls)
        obj.stream = _default_stream() if stream is None else stream
        h = _h()
        rc = lib.mps_load(ctypes.byref(h), os.fsencode(path), obj.stream)
        if rc != MPS_OK:
            raise MPSError(rc, f"mps_load failed for {path}")
        obj._h = h
        L, d, N, chi, prec = (ctypes.c_int() for _ in range(5))
        lib.mps_info(h, ctypes.byref(L), ctypes.byref(d), ctypes.byref(N), ctypes.byref(chi), ctypes.byref(prec))
        obj.L, obj.d, obj.N, obj.chi_max = L.value, d.value, N.value, chi.value
        zn, nc = ctypes.c_int(0), ctypes.c_int(0)
        q = np.zeros(4 * MPS_MAX_D, np.int32)
        lib.mps_charge_rule(h, ctypes.byref(zn), ctypes.byref(nc), _ptr(q, _i32p))
        obj.zn = zn.value
        if nc.value:
            obj.charges = [tuple(int(x) for x in q[i * nc.value:(i + 1) * nc.value]) for i in range(obj.d)]
            obj._set_multi_keys()
            obj.N = obj._dec(obj.N)
        return obj

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib.mps_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def _check(self, rc: int, what: str):
        if rc == MPS_OK:
            return
        msg = lib.mps_last_error(self._h).decode()
        if rc == MPS_ENOCONV:
            warnings.warn(f"{what}: {msg}", JacobiNotConverged)
            return
        raise MPSError(rc, f"{what}: {msg}")

    # -- updates ----------------------------------------------------------------
    def apply_gate2(self, site: int, gate, chi: int, cutoff: float) -> float:
        g = self._gate_flat(gate)
        if g.size != self.gate_length():
            raise ValueError("gate has the wrong number of entries")
        te = ctypes.c_double(0.0)
        rc = lib.mps_apply_gate2(self._h, site, g.ctypes.data_as(_dblp), chi, cutoff, ctypes.byref(te))
        self._check(rc, "mps_apply_gate2")
        return te.value

    def apply_layer(self, sites, gates, chi: int, cutoff: float) -> np.ndarray:
        sites = np.ascontiguousarray(np.asarray(sites, dtype=np.intc))
        gs = [self._gate_flat(g) for g in gates]
        if len(gs) != len(sites):
            raise ValueError("one gate per site")
        if any(g.size != self.gate_length() for g in gs):
            raise ValueError("a gate has the wrong number of entries")
        arr = (_dblp * len(gs))(*[g.ctypes.data_as(_dblp) for g in gs])
        te = np.zeros(len(gs))
        rc = lib.mps_apply_layer(self._h, len(gs), _ptr(sites, _intp), arr, chi, cutoff, _ptr(te, _dblp))
        self._check(rc, "mps_apply_layer")
        return te

    # -- measurements -----------------------------------------------------------
    def expect(self, site: int, diag_op) -> float:
        op = np.ascontiguousarray(np.asarray(diag_op, dtype=np.float64))
        out = ctypes.c_double(0.0)
        self._check(lib.mps_expect(self._h, site, _ptr(op, _dblp), ctypes.byref(out)), "mps_expect")
        return out.value

    def amplitude(self, config) -> complex:
        c = _i32(config)
        out = np.zeros(2)
        self._check(lib.mps_amplitude(self._h, _ptr(c, _i32p), _ptr(out, _dblp)), "mps_amplitude")
        return complex(out[0], out[1])

    def amplitudes(self, configs) -> np.ndarray:
        c = _i32(configs).reshape(-1, self.L)
        out = np.zeros((len(c), 2))
        self._check(lib.mps_amplitude_batch(self._h, len(c), _ptr(c, _i32p), _ptr(out, _dblp)),
                    "mps_amplitude_batch")
        return out[:, 0] + 1j * out[:, 1]

    def sample(self, uniforms):
        """Patterns drawn by sequential conditional sampling (mps_sample) with the given
        n x L uniform numbers in [0, 1); returns (patterns (n, L) int32, probabilities (n,))."""
        u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64)).reshape(-1, self.L)
        n = len(u)
        cfg = np.zeros((n, self.L), np.int32)
        pr = np.zeros(n)
        self._check(lib.mps_sample(self._h, n, _ptr(u, _dblp), _ptr(cfg, _i32p), _ptr(pr, _dblp)), "mps_sample")
        return cfg, pr

    def bond(self, b: int):
        """(charges, dims, lambda per charge) of bond b."""
        n = ctypes.c_int(0)
        cap = self.L * (self.d - 1) + 2 if self.charges is None else min(1 << 16, (self.L + 2) ** len(self.charges[0]))
        ch = np.zeros(cap, np.int32)
        dm = np.zeros(cap, np.int32)
        lam = np.zeros(max(1, self.chi_max) + 1)
        self._check(lib.mps_bond_spectrum(self._h, b, _ptr(ch, _i32p), _ptr(dm, _i32p), _ptr(lam, _dblp), cap,
                                          ctypes.byref(n)), "mps_bond_spectrum")
        k = n.value
        out, off = {}, 0
        for c, D in zip(ch[:k], dm[:k]):
            out[self._dec(c)] = lam[off:off + D].copy()
            off += int(D)
        return out

    def bond_dims(self, b: int) -> dict:
        return {c: len(v) for c, v in self.bond(b).items()}

    def entropy(self, b: int) -> float:
        """Bond entropy -sum lambda^2 ln lambda^2 of bond b (computed by the library)."""
        out = ctypes.c_double(0.0)
        self._check(lib.mps_bond_entropy(self._h, b, ctypes.byref(out)), "mps_bond_entropy")
        return out.value

    def site(self, s: int) -> dict:
        """{(l, m): block} of site s (host copy)."""
        nb, nv = ctypes.c_int(0), ctypes.c_int64(0)
        lib.mps_get_site(self._h, s, None, None, 0, None, 0, ctypes.byref(nb), ctypes.byref(nv))
        lc = np.zeros(max(1, nb.value), np.int32)
        mc = np.zeros(max(1, nb.value), np.int32)
        data = np.zeros(max(1, nv.value), np.complex128)
        rc = lib.mps_get_site(self._h, s, _ptr(lc, _i32p), _ptr(mc, _i32p), nb.value,
                              data.ctypes.data_as(_dblp), nv.value, ctypes.byref(nb), ctypes.byref(nv))
        self._check(rc, "mps_get_site")
        left = self.bond_dims(s)
        right = self.bond_dims(s + 1)
        out, off = {}, 0
        for l, m in zip(lc[:nb.value], mc[:nb.value]):
            l, m = self._dec(l), self._dec(m)
            Dl, Dm = left[l], right[m]
            out[(l, m)] = data[off:off + Dl * Dm].reshape(Dl, Dm).copy()
            off += Dl * Dm
        return out

    def set_bond(self, b: int, lam: dict):
        keys = sorted(lam)
        ch = _i32([self._enc(c) for c in keys])
        dm = _i32([len(lam[c]) for c in keys])
        vals = np.ascontiguousarray(np.concatenate([np.asarray(lam[c], np.float64) for c in keys]))
        self._check(lib.mps_set_bond(self._h, b, len(ch), _ptr(ch, _i32p), _ptr(dm, _i32p), _ptr(vals, _dblp)),
                    "mps_set_bond")

    def set_site(self, s: int, blocks: dict):
        keys = sorted(blocks)
        lc = _i32([self._enc(k[0]) for k in keys])
        mc = _i32([self._enc(k[1]) for k in keys])
        if keys:
            data = np.ascontiguousarray(np.concatenate([np.asarray(blocks[k], np.complex128).reshape(-1)
                                                        for k in keys]))
        else:
            data = np.zeros(1, np.complex128)
        self._check(lib.mps_set_site(self._h, s, len(keys), _ptr(lc, _i32p), _ptr(mc, _i32p),
                                     data.ctypes.data_as(_dblp)), "mps_set_site")

    def batch_sweeps(self) -> dict:
        """Jacobi sweeps of the last update call: sectors, mean and max."""
        n, tot, mx = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        lib.mps_last_batch_sweeps(self._h, ctypes.byref(n), ctypes.byref(tot), ctypes.byref(mx))
        return dict(sectors=n.value, mean=tot.value / max(n.value, 1), max=mx.value)

    def set_profiling(self, on: bool = True):
        self._check(lib.mps_set_profiling(self._h, int(bool(on))), "mps_set_profiling")

    def kernel_stats(self) -> dict:
        """{kind: dict(launches, ms, flops, bytes)} accumulated since the last reset."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            n = ctypes.c_int64()
            ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            self._check(lib.mps_kernel_stats(self._h, k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                             ctypes.byref(by)), "mps_kernel_stats")
            out[name] = dict(launches=n.value, ms=ms.value, flops=fl.value, bytes=by.value)
        return out

    def reset_kernel_stats(self):
        self._check(lib.mps_reset_kernel_stats(self._h), "mps_reset_kernel_stats")

    def set_sweep_limit(self, max_sweeps: int):
        """Jacobi sweep limit (1..40) of this handle's update calls (mps_set_sweep_limit)."""
        self._check(lib.mps_set_sweep_limit(self._h, int(max_sweeps)), "mps_set_sweep_limit")

    def set_chi_deflation(self, level: float = 3e-4):
        """Second SVD deflation level of this handle's updates (0: off; at most 6e-4)."""
        self._check(lib.mps_set_chi_deflation(self._h, float(level)), "mps_set_chi_deflation")

    def deflation_stats(self) -> dict:
        """Updates that deflated their SVDs from the bond's previous cut, and those redone."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(lib.mps_deflation_stats(self._h, ctypes.byref(a), ctypes.byref(b)), "mps_deflation_stats")
        return dict(deflated_updates=a.value, redos=b.value)

    def set_graphs(self, on: bool = True):
        """Capture each update call's launch phases into CUDA graphs (mps_set_graphs)."""
        self._check(lib.mps_set_graphs(self._h, int(bool(on))), "mps_set_graphs")

    def graph_stats(self) -> dict:
        return _graph_stats(self._h)

    def set_autotune(self, on: bool = True):
        """Choose the SVD tile shape per sector-size histogram (mps_set_autotune)."""
        self._check(lib.mps_set_autotune(self._h, int(bool(on))), "mps_set_autotune")

    # -- ground states ----------------------------------------------------------
    def dmrg(self, bond_terms, n_sweeps: int, chi: int, cutoff: float, lanczos_dim: int = 24,
             tol: float = 1e-12) -> np.ndarray:
        """Two-site DMRG sweeps (mps_dmrg); bond_terms[k] holds the charge blocks of h_{k,k+1}.

        Returns the Lanczos eigenvalue of every local step."""
        hs = [_c128_flat(h) for h in bond_terms]
        if len(hs) != self.L - 1:
            raise ValueError("one bond term per bond (L - 1)")
        if any(h.size != gate_length(self.d) for h in hs):
            raise ValueError("a bond term has the wrong number of entries")
        arr = (_dblp * len(hs))(*[h.ctypes.data_as(_dblp) for h in hs])
        cap = n_sweeps * 2 * (self.L - 1)
        en = np.zeros(max(cap, 1))
        n = ctypes.c_int(0)
        rc = lib.mps_dmrg(self._h, arr, n_sweeps, chi, cutoff, lanczos_dim, tol, _ptr(en, _dblp), cap,
                          ctypes.byref(n))
        self._check(rc, "mps_dmrg")
        return en[:n.value].copy()

    def tdvp(self, bond_terms, n_steps: int, dt: float, chi: int, cutoff: float, krylov_dim: int = 24,
             tol: float = 1e-12) -> np.ndarray:
        """Second-order two-site TDVP steps of length dt (mps_tdvp); returns <H_eff> before each
        forward evolution of a pair."""
        hs = [_c128_flat(h) for h in bond_terms]
        if len(hs) != self.L - 1:
            raise ValueError("one bond term per bond (L - 1)")
        if any(h.size != gate_length(self.d) for h in hs):
            raise ValueError("a bond term has the wrong number of entries")
        arr = (_dblp * len(hs))(*[h.ctypes.data_as(_dblp) for h in hs])
        cap = n_steps * 2 * (self.L - 1)
        en = np.zeros(max(cap, 1))
        n = ctypes.c_int(0)
        rc = lib.mps_tdvp(self._h, arr, n_steps, dt, chi, cutoff, krylov_dim, tol, _ptr(en, _dblp), cap,
                          ctypes.byref(n))
        self._check(rc, "mps_tdvp")
        return en[:n.value].copy()

    def dmrg_stats(self) -> dict:
        """Per-kind launches, device ms (with profiling on) and flops of the last dmrg call."""
        out = {}
        for k, name in enumerate(DMRG_KINDS):
            la, ms, fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            lib.mps_dmrg_stats(self._h, k, ctypes.byref(la), ctypes.byref(ms), ctypes.byref(fl))
            out[name] = dict(launches=la.value, ms=ms.value, flops=fl.value)
        mv, rs = ctypes.c_int64(), ctypes.c_int64()
        lib.mps_dmrg_counts(self._h, ctypes.byref(mv), ctypes.byref(rs))
        out["matvecs"], out["lanczos_cycles"] = mv.value, rs.value
        return out

    def stats(self) -> dict:
        a, b, c, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        na, nk = ctypes.c_double(), ctypes.c_double()
        lib.mps_last_update_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(t),
                                  ctypes.byref(na), ctypes.byref(nk))
        return dict(n_sectors=a.value, n_triples=b.value, max_sweeps=c.value, tie_band=t.value,
                    norm_all=na.value, norm_kept=nk.value)


class Executor:
    """Merged updates across handles on one workspace and stream (mps_exec_*)."""

    def __init__(self, stream=None):
        self.stream = _default_stream() if stream is None else stream
        h = _h()
        rc = lib.mps_exec_create(ctypes.byref(h), self.stream)
        if rc != MPS_OK:
            raise MPSError(rc, "mps_exec_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib.mps_exec_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_graphs(self, on: bool = True):
        rc = lib.mps_set_graphs(self._h, int(bool(on)))
        if rc != MPS_OK:
            raise MPSError(rc, "mps_set_graphs")

    def graph_stats(self) -> dict:
        return _graph_stats(self._h)

    def set_autotune(self, on: bool = True):
        rc = lib.mps_set_autotune(self._h, int(bool(on)))
        if rc != MPS_OK:
            raise MPSError(rc, "mps_set_autotune")

    def apply(self, items):
        """items = [(mps, site, flat_gate, chi, cutoff), ...]; returns (trunc_err, status) arrays."""
        n = len(items)
        if n == 0:
            return np.zeros(0), np.zeros(0, dtype=np.intc)
        hs = (_h * n)(*[it[0].handle for it in items])
        sites = np.array([it[1] for it in items], dtype=np.intc)
        gs = [_c128_flat(it[2]) for it in items]
        if any(g.size != it[0].gate_length() for g, it in zip(gs, items)):
            raise ValueError("a gate has the wrong number of entries")
        garr = (_dblp * n)(*[g.ctypes.data_as(_dblp) for g in gs])
        chis = np.array([it[3] for it in items], dtype=np.intc)
        cuts = np.array([it[4] for it in items], dtype=np.float64)
        te = np.zeros(n)
        st = np.zeros(n, dtype=np.intc)
        rc = lib.mps_exec_apply(self._h, n, hs, _ptr(sites, _intp), garr, _ptr(chis, _intp), _ptr(cuts, _dblp),
                                _ptr(te, _dblp), _ptr(st, _intp))
        if rc not in (MPS_OK, MPS_ENOCONV):
            raise MPSError(rc, "mps_exec_apply: " + lib.mps_last_error(self._h).decode())
        return te, st


def _graph_stats(h) -> dict:
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib.mps_graph_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return dict(launches=a.value, updates=b.value, instantiations=c.value)


def autotune_stats() -> dict:
    """Process-wide SVD tile-shape table: keys, tuning runs, reuses."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib.mps_autotune_stats(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return dict(keys=a.value, tuning_runs=b.value, hits=c.value)


def autotune_table() -> str:
    n = ctypes.c_int()
    lib.mps_autotune_table(None, 0, ctypes.byref(n))
    buf = ctypes.create_string_buffer(n.value + 1)
    rc = lib.mps_autotune_table(buf, n.value + 1, ctypes.byref(n))
    if rc != MPS_OK:
        raise MPSError(rc, "mps_autotune_table")
    return buf.value.decode()


def autotune_clear() -> None:
    lib.mps_autotune_clear()


def tc_inject_stall(on: bool) -> None:
    """Tensor-core GEMMs launched afterwards issue no MMA and report a bounded-wait expiry."""
    lib.mps_tc_inject_stall(int(bool(on)))


def autotune_force(candidate: int) -> None:
    """Every update call uses SVD tile-shape candidate 0..9 (-1: back to normal)."""
    rc = lib.mps_autotune_force(int(candidate))
    if rc != MPS_OK:
        raise MPSError(rc, "mps_autotune_force")


def autotune_freeze(frozen: bool = True) -> None:
    """Frozen: sector-size histograms not yet in the table keep the default shape, untuned."""
    lib.mps_autotune_freeze(int(bool(frozen)))


def svd_mixed_min_k(min_k: int) -> None:
    """Cluster SVD sectors with min(m, n) >= min_k start with FP32 Jacobi sweeps (0: off)."""
    rc = lib.mps_svd_mixed_min_k(int(min_k))
    if rc != MPS_OK:
        raise MPSError(rc, "mps_svd_mixed_min_k")


def svd_cluster_min_k(min_k: int) -> None:
    """Sectors with min(m, n) >= min_k use the cluster SVD kernels (0: only those that do not fit one CTA)."""
    rc = lib.mps_svd_cluster_min_k(int(min_k))
    if rc != MPS_OK:
        raise MPSError(rc, "mps_svd_cluster_min_k")


def svd_mixed_sweeps(max_sweeps: int) -> None:
    """Limit of the FP32 sweeps of the mixed-precision SVD start (1..40)."""
    rc = lib.mps_svd_mixed_sweeps(int(max_sweeps))
    if rc != MPS_OK:
        raise MPSError(rc, "mps_svd_mixed_sweeps")


def autotune_min_flops(flops: float) -> None:
    """Nominal SVD flops below which a batch keeps the default tile shape."""
    rc = lib.mps_autotune_min_flops(float(flops))
    if rc != MPS_OK:
        raise MPSError(rc, "mps_autotune_min_flops")


def footprint_bytes(L: int, d: int, N: int, chi_max: int) -> tuple[int, int]:
    """(arena bytes of a handle, upper bound of one layer's update workspace)."""
    a, w = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.mps_footprint_bytes(L, d, N, chi_max, ctypes.byref(a), ctypes.byref(w))
    if rc != MPS_OK:
        raise MPSError(rc, "mps_footprint_bytes")
    return a.value, w.value


def zgemm_tc(A: np.ndarray, B: np.ndarray, precision: int = MPS_TF32, stream=None) -> np.ndarray:
    """C = A B (complex) on the tensor cores through mps_zgemm_tc; torch holds the device buffers."""
    import torch
    A = np.ascontiguousarray(A, np.complex128)
    B = np.ascontiguousarray(B, np.complex128)
    M, K = A.shape
    K2, N = B.shape
    if K2 != K:
        raise ValueError("inner dimensions differ")
    dev = torch.device("cuda")
    dA = torch.from_numpy(A.view(np.float64).copy()).to(dev)
    dB = torch.from_numpy(B.view(np.float64).copy()).to(dev)
    dC = torch.zeros(2 * M * N, dtype=torch.float64, device=dev)
    wb = int(lib.mps_zgemm_tc_work_bytes(precision, M, N, K))
    if wb < 0:
        raise MPSError(MPS_EINVAL, "mps_zgemm_tc_work_bytes")
    dW = torch.zeros(wb, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    rc = lib.mps_zgemm_tc(precision, M, N, K, dA.data_ptr(), K, dB.data_ptr(), N, dC.data_ptr(), N, dW.data_ptr(),
                          wb, st)
    if rc != MPS_OK:
        raise MPSError(rc, "mps_zgemm_tc")
    return dC.cpu().numpy().view(np.complex128).reshape(M, N)


def fp64_peak_probe(stream=None) -> float:
    """Measured FP64 FMA throughput of the current GPU, GFLOP/s."""
    g = ctypes.c_double()
    rc = lib.mps_fp64_peak_probe(ctypes.byref(g), _default_stream() if stream is None else stream)
    if rc != MPS_OK:
        raise MPSError(rc, "mps_fp64_peak_probe")
    return g.value


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib.mps_launch_count())


def apply_gate2_batch(items, stream_owner: MPS | None = None):
    """Merged updates across handles: items = [(mps, site, gate, chi, cutoff), ...]."""
    n = len(items)
    hs = (_h * n)(*[it[0].handle for it in items])
    sites = np.array([it[1] for it in items], dtype=np.intc)
    gs = [it[0]._gate_flat(it[2]) for it in items]
    if any(g.size != it[0].gate_length() for g, it in zip(gs, items)):
        raise ValueError("a gate has the wrong number of entries")
    garr = (_dblp * n)(*[g.ctypes.data_as(_dblp) for g in gs])
    chis = np.array([it[3] for it in items], dtype=np.intc)
    cuts = np.array([it[4] for it in items], dtype=np.float64)
    te = np.zeros(n)
    st = np.zeros(n, dtype=np.intc)
    rc = lib.mps_apply_gate2_batch(n, hs, _ptr(sites, _intp), garr, _ptr(chis, _intp), _ptr(cuts, _dblp),
                                   _ptr(te, _dblp), _ptr(st, _intp))
    if rc not in (MPS_OK, MPS_ENOCONV):
        raise MPSError(rc, "mps_apply_gate2_batch: " + lib.mps_last_error(items[0][0].handle).decode())
    return te, st


def plan_sectors(d: int, left: dict, mid: dict, right: dict):
    """The library's integer sector planner: (triples, sectors) as int arrays."""
    def tab(t):
        ks = sorted(t)
        return _i32(ks), _i32([t[k] for k in ks])
    (lc, ld), (mc, md), (rc, rd) = tab(left), tab(mid), tab(right)
    cap_t = max(1, len(lc) * len(mc) * len(rc))
    cap_s = max(1, len(lc) + len(rc) + 2 * d)
    tri = np.zeros(3 * cap_t, np.int32)
    sec = np.zeros(3 * cap_s, np.int32)
    nt, ns = ctypes.c_int(), ctypes.c_int()
    rcode = lib.mps_plan_sectors(d, len(lc), _ptr(lc, _i32p), _ptr(ld, _i32p), len(mc), _ptr(mc, _i32p),
                                 _ptr(md, _i32p), len(rc), _ptr(rc, _i32p), _ptr(rd, _i32p), _ptr(tri, _i32p),
                                 cap_t, ctypes.byref(nt), _ptr(sec, _i32p), cap_s, ctypes.byref(ns))
    if rcode != MPS_OK:
        raise MPSError(rcode, "mps_plan_sectors")
    return tri[:3 * nt.value].reshape(-1, 3), sec[:3 * ns.value].reshape(-1, 3)


def plan_sectors_rule(d: int, left: dict, mid: dict, right: dict, zn: int = 0, charges=None, radix=None):
    """The library's sector planner under any charge rule (mps_plan_sectors_rule).

    zn: n of a Z_n rule (d <= n).  charges: d charge vectors of a several-U(1) rule, with the
    tables keyed by charge tuples and radix the mixed radix of their encoding (default: each
    component's radix 2 * (largest table value) + 3).  Returns (triples, sectors) with
    triples a list of (l, m, r) and sectors a list of (c, rows, cols, row charges, column
    charges), charges as tuples for a several-U(1) rule.
    """
    ncomp = 0 if charges is None else len(charges[0])
    if ncomp:
        if radix is None:
            top = [max([0] + [int(k[j]) for t in (left, mid, right) for k in t]) for j in range(ncomp)]
            radix = [2 * t + 3 for t in top]
        weights = [int(np.prod(radix[j + 1:])) for j in range(ncomp)]
        enc = lambda c: int(sum(int(x) * w for x, w in zip(c, weights)))

        def dec(v):
            out = []
            for w in weights:
                out.append(int(v) // w)
                v = int(v) - out[-1] * w
            return tuple(out)
        q = _i32([x for vec in charges for x in vec])
        rad = _i32(radix)
    else:
        enc = dec = int
        q = rad = None

    def tab(t):
        ks = sorted(t, key=enc)
        return _i32([enc(k) for k in ks]), _i32([t[k] for k in ks])
    (lc, ld), (mc, md), (rc, rd) = tab(left), tab(mid), tab(right)
    cap_t = max(1, len(lc) * len(mc) * len(rc))
    cap_s = max(1, len(lc) * len(rc) * d + 2 * d)
    cap_l = max(1, cap_s * (len(lc) + len(rc)))
    tri = np.zeros(3 * cap_t, np.int32)
    sec = np.zeros(5 * cap_s, np.int32)
    lst = np.zeros(cap_l, np.int32)
    nt, ns, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rcode = lib.mps_plan_sectors_rule(d, zn, ncomp, None if q is None else _ptr(q, _i32p),
                                      None if rad is None else _ptr(rad, _i32p),
                                      len(lc), _ptr(lc, _i32p), _ptr(ld, _i32p), len(mc), _ptr(mc, _i32p),
                                      _ptr(md, _i32p), len(rc), _ptr(rc, _i32p), _ptr(rd, _i32p),
                                      _ptr(tri, _i32p), cap_t, ctypes.byref(nt), _ptr(sec, _i32p), cap_s,
                                      ctypes.byref(ns), _ptr(lst, _i32p), cap_l, ctypes.byref(nl))
    if rcode != MPS_OK:
        raise MPSError(rcode, "mps_plan_sectors_rule")
    triples = [tuple(dec(x) for x in t) for t in tri[:3 * nt.value].reshape(-1, 3).tolist()]
    sectors, o = [], 0
    for c, rows, cols, nr_, nc_ in sec[:5 * ns.value].reshape(-1, 5).tolist():
        rl = [dec(x) for x in lst[o:o + nr_]]
        cl = [dec(x) for x in lst[o + nr_:o + nr_ + nc_]]
        o += nr_ + nc_
        sectors.append((dec(c), rows, cols, rl, cl))
    return triples, sectors


def gate_layout(d: int, zn: int = 0, charges=None):
    """The library's gate layout of a charge rule (mps_gate_layout): (block sizes, length)."""
    nc = 0 if charges is None else len(charges[0])
    q = None if charges is None else _i32([x for vec in charges for x in vec])
    sizes = np.zeros(4 * MPS_MAX_D * MPS_MAX_D, np.int32)
    nb, ln = ctypes.c_int(0), ctypes.c_int64(0)
    rc = lib.mps_gate_layout(d, zn, nc, None if q is None else _ptr(q, _i32p), _ptr(sizes, _i32p), len(sizes),
                             ctypes.byref(nb), ctypes.byref(ln))
    if rc != MPS_OK:
        raise MPSError(rc, "mps_gate_layout")
    return [int(x) for x in sizes[:nb.value]], int(ln.value)


def svd_work_bytes(ms, ns) -> int:
    m = np.ascontiguousarray(np.asarray(ms, dtype=np.intc))
    n = np.ascontiguousarray(np.asarray(ns, dtype=np.intc))
    return int(lib.mps_svd_work_bytes(len(m), _ptr(m, _intp), _ptr(n, _intp)))


def svd_sectors(mats, rowscales=None, stream=None):
    """Batched sector SVD on the GPU through mps_svd_sectors (torch supplies device memory).

    mats: list of complex128 host arrays (m_k x n_k).  Returns [(sigma, Y, sweeps)] with
    M_k = diag(rowscale_k) mats_k = X S Y^dag.
    """
    import torch
    dev = torch.device("cuda")
    ms = [a.shape[0] for a in mats]
    ns = [a.shape[1] for a in mats]
    ks = [min(a, b) for a, b in zip(ms, ns)]
    mat_off = np.cumsum([0] + [a * b for a, b in zip(ms, ns)])[:-1].astype(np.int64)
    y_off = np.cumsum([0] + [n * k for n, k in zip(ns, ks)])[:-1].astype(np.int64)
    s_off = np.cumsum([0] + ks)[:-1].astype(np.int64)
    r_off = np.cumsum([0] + ms)[:-1].astype(np.int64)
    flat = np.concatenate([np.ascontiguousarray(a, np.complex128).reshape(-1) for a in mats])
    d_mats = torch.from_numpy(flat.view(np.float64).copy()).to(dev)
    d_sig = torch.zeros(sum(ks), dtype=torch.float64, device=dev)
    d_y = torch.zeros(2 * sum(n * k for n, k in zip(ns, ks)), dtype=torch.float64, device=dev)
    d_st = torch.zeros(len(mats), dtype=torch.int32, device=dev)
    wb = svd_work_bytes(ms, ns)
    d_work = torch.zeros(max(wb, 256), dtype=torch.uint8, device=dev)
    d_rs = None
    if rowscales is not None:
        d_rs = torch.from_numpy(np.concatenate([np.asarray(r, np.float64) for r in rowscales])).to(dev)
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    m_a = np.asarray(ms, np.intc)
    n_a = np.asarray(ns, np.intc)
    rc = lib.mps_svd_sectors(len(mats), _ptr(m_a, _intp), _ptr(n_a, _intp), d_mats.data_ptr(),
                             _ptr(mat_off, _i64p), d_rs.data_ptr() if d_rs is not None else None,
                             _ptr(r_off, _i64p) if d_rs is not None else None,
                             d_sig.data_ptr(), _ptr(s_off, _i64p), d_y.data_ptr(), _ptr(y_off, _i64p),
                             d_st.data_ptr(), d_work.data_ptr(), d_work.numel(), st)
    if rc != MPS_OK:
        raise MPSError(rc, "mps_svd_sectors")
    torch.cuda.synchronize()
    sig = d_sig.cpu().numpy()
    y = d_y.cpu().numpy().view(np.complex128)
    sts = d_st.cpu().numpy()
    out = []
    for k in range(len(mats)):
        Y = y[y_off[k]:y_off[k] + ns[k] * ks[k]].reshape(ks[k], ns[k]).T   # column-major n x k
        out.append((sig[s_off[k]:s_off[k] + ks[k]].copy(), Y.copy(), int(sts[k])))
    return out


def svd_sectors_noalloc(mats, rowscales=None, stream=None):
    """The same batched sector SVD through mps_svd_sectors_noalloc.

    For callers that must not allocate device memory: no scratch buffer is passed
    and the library allocates nothing (its scratch is a fixed device array of
    MPS_NOALLOC_SCRATCH_BYTES).  torch holds only the inputs and outputs here.
    Returns [(sigma, Y, sweeps)] like svd_sectors.
    """
    import torch
    dev = torch.device("cuda")
    ms = [a.shape[0] for a in mats]
    ns = [a.shape[1] for a in mats]
    ks = [min(a, b) for a, b in zip(ms, ns)]
    mat_off = np.cumsum([0] + [a * b for a, b in zip(ms, ns)])[:-1].astype(np.int64)
    y_off = np.cumsum([0] + [n * k for n, k in zip(ns, ks)])[:-1].astype(np.int64)
    s_off = np.cumsum([0] + ks)[:-1].astype(np.int64)
    r_off = np.cumsum([0] + ms)[:-1].astype(np.int64)
    flat = np.concatenate([np.ascontiguousarray(a, np.complex128).reshape(-1) for a in mats])
    d_mats = torch.from_numpy(flat.view(np.float64).copy()).to(dev)
    d_sig = torch.zeros(sum(ks), dtype=torch.float64, device=dev)
    d_y = torch.zeros(2 * sum(n * k for n, k in zip(ns, ks)), dtype=torch.float64, device=dev)
    d_st = torch.zeros(len(mats), dtype=torch.int32, device=dev)
    d_rs = None
    if rowscales is not None:
        d_rs = torch.from_numpy(np.concatenate([np.asarray(r, np.float64) for r in rowscales])).to(dev)
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    m_a = np.asarray(ms, np.intc)
    n_a = np.asarray(ns, np.intc)
    rc = lib.mps_svd_sectors_noalloc(len(mats), _ptr(m_a, _intp), _ptr(n_a, _intp), d_mats.data_ptr(),
                                     _ptr(mat_off, _i64p), d_rs.data_ptr() if d_rs is not None else None,
                                     _ptr(r_off, _i64p) if d_rs is not None else None,
                                     d_sig.data_ptr(), _ptr(s_off, _i64p), d_y.data_ptr(), _ptr(y_off, _i64p),
                                     d_st.data_ptr(), st)
    if rc != MPS_OK:
        raise MPSError(rc, "mps_svd_sectors_noalloc")
    torch.cuda.synchronize()
    sig = d_sig.cpu().numpy()
    y = d_y.cpu().numpy().view(np.complex128)
    sts = d_st.cpu().numpy()
    out = []
    for k in range(len(mats)):
        Y = y[y_off[k]:y_off[k] + ns[k] * ks[k]].reshape(ks[k], ns[k]).T
        out.append((sig[s_off[k]:s_off[k] + ks[k]].copy(), Y.copy(), int(sts[k])))
    return out
