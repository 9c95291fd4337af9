"""ctypes binding of librs (include/rs.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts
Python polynomials to the C structs and results back.  There is no fallback:
if ``librs.so`` is missing or cannot be loaded, ``load()`` raises.
"""
import ctypes
import math
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int32, c_int64, c_uint32, c_void_p

import numpy as np

from .inputs import BiPoly

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librs.so")

RS_OK, RS_PENDING = 0, 1
ERRORS = {-1: "RS_ERR_ARG", -2: "RS_ERR_CAPACITY", -3: "RS_ERR_NOMEM", -4: "RS_ERR_CUDA",
          -5: "RS_ERR_TIMEOUT", -6: "RS_ERR_LIMIT", -7: "RS_ERR_STATE"}
RS_MAX_LIMBS, RS_MAX_DEG_Y, RS_MAX_POINTS, RS_MAX_PRIMES = 128, 71, 16384, 16384

# Every function that include/rs.h declares, with its ctypes signature.
EXPORTS = {}


class rs_bipoly(ctypes.Structure):
    _fields_ = [("deg_x", c_int32), ("deg_y", c_int32), ("limbs", c_int32),
                ("coeffs", POINTER(c_uint32))]


class rs_upoly(ctypes.Structure):
    _fields_ = [("deg", c_int32), ("limbs", c_int32), ("capacity_words", c_int64),
                ("coeffs", POINTER(c_uint32))]


class rs_config(ctypes.Structure):
    _fields_ = [("device", c_int32), ("tile_points", c_int32), ("use_graphs", c_int32),
                ("persistent", c_int32), ("timing", c_int32), ("autotune", c_int32),
                ("g2_form", c_int32), ("univariate", c_int32),
                ("mem_limit_bytes", c_int64), ("autotune_cache", c_char_p),
                ("crt_form", c_int32), ("reserved", c_int32)]


class rs_tune_entry(ctypes.Structure):
    _fields_ = [(k, c_int32) for k in ("kind", "sms", "cap", "lg_points", "lg_images", "choice",
                                       "persistent")] + [("ms_best", ctypes.c_float),
                                                         ("ms_default", ctypes.c_float)]


class rs_batch_info(ctypes.Structure):
    _fields_ = [("pairs", c_int64), ("images", c_int64), ("primes_total", c_int64),
                ("coeffs_total", c_int64), ("modmul_eval", c_double), ("modmul_prs", c_double),
                ("modmul_interp", c_double), ("modmul_crt", c_double), ("input_bytes", c_int64),
                ("output_bytes", c_int64), ("ms_images", c_float), ("ms_interp", c_float),
                ("ms_crt", c_float), ("ms_total", c_float), ("unlucky_points", c_int64),
                ("degenerate_images", c_int64), ("unlucky_primes", c_int64),
                ("kernel_launches", c_int64), ("ms_yun", c_float), ("reserved", c_int32)]


class rs_sqf_info(ctypes.Structure):
    _fields_ = [("batch", rs_batch_info), ("yun_tasks", c_int64), ("factors", c_int64),
                ("ms_lift", c_float), ("ms_host", c_float), ("ms_total", c_float),
                ("ms_primitive", c_float), ("h2d_bytes", c_int64), ("d2h_bytes", c_int64),
                ("ms_analyse", c_float), ("ms_contents", c_float), ("ms_fetch", c_float),
                ("factors_device", c_int32)]


class rs_server_stats(ctypes.Structure):
    _fields_ = [(n, c_int64) for n in ("submitted", "completed", "failed", "pending", "running",
                                        "inflight_batches", "batches", "peak_inflight_batches",
                                        "peak_running", "mem_used", "mem_limit",
                                        "kernel_launches")]


class rs_int_peak(ctypes.Structure):
    _fields_ = [(n, c_double) for n in ("mad_lo_u32", "mad_wide_u32", "mad_hi_u32", "mad_wide_s32",
                                         "mont_update", "clock_max_mhz")] + \
               [("sms", c_int32), ("launches", c_int32)]


_P = POINTER
_SIGS = {
    "rs_measure_int_peak": (c_int32, [_P(rs_int_peak)]),
    "rs_config_default": (c_int32, [_P(rs_config)]),
    "rs_create": (c_int32, [_P(c_void_p), _P(rs_config)]),
    "rs_destroy": (c_int32, [c_void_p]),
    "rs_stream": (c_int32, [c_void_p, _P(c_void_p)]),
    "rs_error_string": (c_char_p, [c_int32]),
    "rs_last_error": (c_char_p, [c_void_p]),
    "rs_result_bound": (c_int32, [_P(rs_bipoly), _P(rs_bipoly), _P(c_int32), _P(c_int32),
                                  _P(c_int32), _P(c_int32)]),
    "rs_resultant_y": (c_int32, [c_void_p, _P(rs_bipoly), _P(rs_bipoly), _P(rs_upoly)]),
    "rs_resultant_batch": (c_int32, [c_void_p, c_int32, _P(rs_bipoly), _P(rs_bipoly),
                                     _P(rs_upoly), _P(c_int32)]),
    "rs_batch_create": (c_int32, [c_void_p, c_int32, _P(rs_bipoly), _P(rs_bipoly), _P(c_void_p)]),
    "rs_batch_create_on": (c_int32, [c_void_p, c_int32, _P(rs_bipoly), _P(rs_bipoly), c_void_p,
                                     _P(c_void_p)]),
    "rs_batch_upload": (c_int32, [c_void_p, c_int32, _P(rs_bipoly), _P(rs_bipoly)]),
    "rs_batch_run": (c_int32, [c_void_p]),
    "rs_batch_sync": (c_int32, [c_void_p]),
    "rs_batch_results": (c_int32, [c_void_p, _P(rs_upoly), _P(c_int32)]),
    "rs_batch_destroy": (c_int32, [c_void_p]),
    "rs_batch_info_get": (c_int32, [c_void_p, _P(rs_batch_info)]),
    "rs_images": (c_int32, [c_void_p, _P(rs_bipoly), _P(rs_bipoly), c_int32, c_int32,
                            _P(c_uint32), _P(c_uint32), _P(c_uint32)]),
    "rs_crt_noalloc": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p]),
    "rs_server_start": (c_int32, [c_void_p, c_int32, c_int32, c_int64]),
    "rs_server_submit": (c_int32, [c_void_p, _P(rs_bipoly), _P(rs_bipoly), _P(ctypes.c_uint64)]),
    "rs_server_poll": (c_int32, [c_void_p, ctypes.c_uint64, _P(rs_upoly), _P(c_double)]),
    "rs_server_wait": (c_int32, [c_void_p, ctypes.c_uint64, _P(rs_upoly), _P(c_double), c_int64]),
    "rs_server_stats_get": (c_int32, [c_void_p, _P(rs_server_stats)]),
    "rs_server_stop": (c_int32, [c_void_p]),
    "rs_server_set_log": (c_int32, [c_void_p, c_char_p]),
    "rs_resultant_x": (c_int32, [c_void_p, _P(rs_bipoly), _P(rs_bipoly), _P(rs_upoly)]),
    "rs_projections": (c_int32, [c_void_p, c_int32, _P(rs_bipoly), _P(rs_bipoly), _P(rs_upoly),
                                 _P(rs_upoly), _P(c_int32)]),
    "rs_squarefree_y": (c_int32, [c_void_p, _P(rs_bipoly), _P(rs_bipoly), c_int32, _P(rs_upoly),
                                  _P(rs_upoly), _P(c_int32)]),
    "rs_squarefree_batch": (c_int32, [c_void_p, c_int32, _P(rs_bipoly), _P(rs_bipoly), c_int32,
                                      _P(rs_upoly), _P(rs_upoly), _P(c_int32), _P(c_int32)]),
    "rs_squarefree_info_get": (c_int32, [c_void_p, _P(rs_sqf_info)]),
    "rs_squarefree_projections": (c_int32, [c_void_p, c_int32, _P(rs_bipoly), _P(rs_bipoly), c_int32,
                                            _P(rs_upoly), _P(rs_upoly), _P(c_int32), c_void_p, c_void_p,
                                            c_void_p, _P(c_int32)]),
    "rs_autotune": (c_int32, [c_void_p, c_int32, _P(rs_bipoly), _P(rs_bipoly)]),
    "rs_autotune_entries": (c_int32, [_P(rs_tune_entry), c_int32, _P(c_int32)]),
    "rs_autotune_save": (c_int32, [c_char_p]),
    "rs_autotune_load": (c_int32, [c_char_p]),
    "rs_autotune_clear": (c_int32, []),
    "rs_test_stall_tensor_cores": (c_int32, [c_void_p, c_int32]),
}

_lib = None


def load(path=None):
    """Load librs.so (raises OSError if it is missing: no fallback exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"librs.so not built at {p}; run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
        EXPORTS[name] = fn
    if path is None:
        _lib = lib
    return lib


def measure_int_peak():
    """Integer multiply-add throughputs of the current device (operations per
    second over all SMs): mad.lo.u32, mad.wide.u32, mad.hi.u32, mad.wide.s32
    and the Montgomery remainder step; plus the SM count and max clock."""
    out = rs_int_peak()
    rc = load().rs_measure_int_peak(ctypes.byref(out))
    if rc:
        raise RsError(rc, "rs_measure_int_peak")
    return {n: getattr(out, n) for n, _ in rs_int_peak._fields_}


class RsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(rc, ctx=None):
    if rc < 0:
        lib = load()
        raise RsError(rc, (lib.rs_last_error(ctx) or b"").decode())
    return rc


def as_bipoly(f):
    return f if isinstance(f, BiPoly) else BiPoly.from_ints(f)


# Host image of rs_bipoly (three int32, padding, a pointer), filled with
# vectorised numpy and viewed as the ctypes struct array.
_BIPOLY_DT = np.dtype([("deg_x", "<i4"), ("deg_y", "<i4"), ("limbs", "<i4"), ("pad", "<i4"),
                       ("coeffs", "<u8")])


def _abi_record(b):
    """(limb array, deg_x, deg_y, limbs, 0, data pointer) of a BiPoly, kept on
    the instance while its coefficient array stays the same object, so that
    marshalling the same inputs again costs one attribute lookup each."""
    rec = getattr(b, "_rs_abi", None)
    if rec is None or rec[0] is not b.coeffs:
        a = b.coeffs
        if not (a.dtype == np.uint32 and a.flags.c_contiguous):
            a = np.ascontiguousarray(a, dtype=np.uint32)
            b.coeffs = a
        rec = (a, a.shape[0] - 1, a.shape[1] - 1, a.shape[2], 0, a.__array_interface__["data"][0])
        b._rs_abi = rec
    return rec


class _Polys:
    """Keeps the limb arrays alive while C structs point at them."""

    def __init__(self, polys):
        recs = [_abi_record(as_bipoly(p)) for p in polys]
        n = len(recs)
        self.arrays = [r[0] for r in recs]
        self.raw = np.zeros(max(n, 1), dtype=_BIPOLY_DT)
        if n:
            self.raw[:n] = np.array([r[1:] for r in recs], dtype=_BIPOLY_DT)
        self.structs = (rs_bipoly * max(n, 1)).from_buffer(self.raw)


def swap_xy(f):
    """The same polynomial with x and y exchanged (only used here to size the
    output buffers of Res_x; the library exchanges the variables itself)."""
    b = as_bipoly(f)
    return BiPoly(np.ascontiguousarray(b.coeffs.transpose(1, 0, 2)))


def result_bound(f, g):
    """Host-only planning: degree bound, output limbs, primes, bits."""
    lib = load()
    P = _Polys([f, g])
    d, l, k, b = c_int32(), c_int32(), c_int32(), c_int32()
    _check(lib.rs_result_bound(ctypes.byref(P.structs[0]), ctypes.byref(P.structs[1]),
                               ctypes.byref(d), ctypes.byref(l), ctypes.byref(k), ctypes.byref(b)))
    return {"deg": d.value, "limbs": l.value, "primes": k.value, "bits": b.value}


def limbs_to_ints(words, deg, limbs):
    if deg < 0:
        return []
    w = np.ascontiguousarray(words[: (deg + 1) * limbs]).astype("<u4").reshape(deg + 1, limbs)
    return [int.from_bytes(r.tobytes(), "little", signed=True) for r in w]


class _Outputs:
    def __init__(self, pairs):
        self.bufs = []
        self.structs = (rs_upoly * max(len(pairs), 1))()
        for s, (f, g) in zip(self.structs, pairs):
            b = result_bound(f, g)
            words = max(1, (b["deg"] + 1) * b["limbs"])
            buf = np.zeros(words, dtype=np.uint32)
            self.bufs.append(buf)
            s.capacity_words = words
            s.coeffs = buf.ctypes.data_as(POINTER(c_uint32))

    def ints(self):
        return [limbs_to_ints(b, s.deg, s.limbs) for s, b in zip(self.structs, self.bufs)]

    def raw(self):
        return [(s.deg, s.limbs, b) for s, b in zip(self.structs, self.bufs)]


class Context:
    """One librs context (device memory, stream, prime tables) on one GPU."""

    def __init__(self, device=-1, tile_points=0, use_graphs=True, persistent=True, timing=False,
                 mem_limit_bytes=0, autotune=True, autotune_cache=None, g2_form=0, univariate="prs",
                 crt_form=0):
        """univariate: "prs" (division-free remainder sequence, one thread per
        image) or "schur" (Schur algorithm on displacement generators, one
        warp per image); crt_form: rs_config.crt_form (0 by batch shape, 1
        CUDA cores only, 2 tensor cores where possible)."""
        lib = load()
        cfg = rs_config()
        _check(lib.rs_config_default(ctypes.byref(cfg)))
        cfg.device, cfg.tile_points = device, tile_points
        cfg.use_graphs, cfg.persistent, cfg.timing = int(use_graphs), int(persistent), int(timing)
        cfg.mem_limit_bytes = mem_limit_bytes
        cfg.autotune = int(autotune)
        cfg.g2_form = int(g2_form)
        cfg.crt_form = int(crt_form)
        if univariate not in ("prs", "schur"):
            raise ValueError("univariate must be 'prs' or 'schur'")
        cfg.univariate = 1 if univariate == "schur" else 0
        cfg.autotune_cache = os.fsencode(autotune_cache) if autotune_cache else None
        h = c_void_p()
        _check(lib.rs_create(ctypes.byref(h), ctypes.byref(cfg)))
        self.lib, self.h = lib, h

    def close(self):
        if self.h:
            self.lib.rs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self):
        s = c_void_p()
        _check(self.lib.rs_stream(self.h, ctypes.byref(s)), self.h)
        return s.value or 0

    def stall_tensor_cores(self, on):
        """Test hook: rs_test_stall_tensor_cores (the tensor-core kernels'
        bounded waits run out; runs fail with RS_ERR_TIMEOUT)."""
        _check(self.lib.rs_test_stall_tensor_cores(self.h, int(bool(on))))

    def resultant_y(self, f, g):
        """Res_y(f, g) as a list of Python ints (coefficient of x^i at i)."""
        P = _Polys([f, g])
        out = _Outputs([(f, g)])
        _check(self.lib.rs_resultant_y(self.h, ctypes.byref(P.structs[0]),
                                       ctypes.byref(P.structs[1]), out.structs), self.h)
        return out.ints()[0]

    def resultant_batch(self, pairs, raw=False):
        F, G = _Polys([p[0] for p in pairs]), _Polys([p[1] for p in pairs])
        out = _Outputs(pairs)
        status = (c_int32 * max(len(pairs), 1))()
        _check(self.lib.rs_resultant_batch(self.h, len(pairs), F.structs, G.structs, out.structs,
                                           status), self.h)
        return out.raw() if raw else out.ints()

    def resultant_x(self, f, g):
        """Res_x(f, g) in Z[y] as a list of Python ints (coefficient k of y^k)."""
        P = _Polys([f, g])
        out = _Outputs([(swap_xy(f), swap_xy(g))])
        _check(self.lib.rs_resultant_x(self.h, ctypes.byref(P.structs[0]),
                                       ctypes.byref(P.structs[1]), out.structs), self.h)
        return out.ints()[0]

    def projections(self, pairs, raw=False):
        """(Res_y list, Res_x list) of every pair, computed in one batch."""
        F, G = _Polys([p[0] for p in pairs]), _Polys([p[1] for p in pairs])
        oy = _Outputs(pairs)
        ox = _Outputs([(swap_xy(f), swap_xy(g)) for f, g in pairs])
        status = (c_int32 * max(2 * len(pairs), 1))()
        _check(self.lib.rs_projections(self.h, len(pairs), F.structs, G.structs, oy.structs,
                                       ox.structs, status), self.h)
        if raw:
            return oy.raw(), ox.raw()
        return oy.ints(), ox.ints()

    def squarefree(self, f, g, max_mult=8):
        """Square-free factorisation of Res_y(f, g): (c, [(i, R_i), ...]) with
        Res_y = c * prod R_i^i (R_i as lists of Python ints, ascending; only
        the non-constant factors, in increasing multiplicity)."""
        out = self.squarefree_batch([(f, g)], max_mult)[0]
        if isinstance(out, RsError):
            raise out
        return out

    def squarefree_batch(self, pairs, max_mult=8, raw=False):
        """Square-free factorisations of Res_y(f, g) for every (f, g) in pairs
        in one GPU pass: per pair (c, [(i, R_i), ...]) as squarefree()
        returns, or the RsError of a pair that failed (``raw``: only the
        per-pair status codes; the limbs stay in the host buffers)."""
        n = len(pairs)
        if n == 0:
            return []
        F, G = _Polys([p[0] for p in pairs]), _Polys([p[1] for p in pairs])

        def call(content, facs, nm, st):
            return self.lib.rs_squarefree_batch(self.h, n, F.structs, G.structs, max_mult, content, facs, nm, st)
        return self._squarefree_call(list(pairs), max_mult, call, raw)

    def squarefree_projections(self, pairs, max_mult=8):
        """Square-free factorisations of both projections of every pair in one
        GPU pass: per pair (sqf of Res_y, sqf of Res_x), each as squarefree()
        returns (Res_x's coefficient k belongs to y^k) or an RsError."""
        n = len(pairs)
        if n == 0:
            return []
        F, G = _Polys([p[0] for p in pairs]), _Polys([p[1] for p in pairs])
        sz_u, sz_i = ctypes.sizeof(rs_upoly), ctypes.sizeof(c_int32)

        def call(content, facs, nm, st):
            return self.lib.rs_squarefree_projections(
                self.h, n, F.structs, G.structs, max_mult, content, facs, nm,
                c_void_p(ctypes.addressof(content) + n * sz_u),
                c_void_p(ctypes.addressof(facs) + n * max_mult * sz_u),
                c_void_p(ctypes.addressof(nm) + n * sz_i), st)
        sizing = list(pairs) + [(swap_xy(f), swap_xy(g)) for f, g in pairs]
        out = self._squarefree_call(sizing, max_mult, call, False)
        return list(zip(out[:n], out[n:]))

    def _squarefree_call(self, pairs, max_mult, call, raw):
        """Size the output buffers of len(pairs) factorisations from the
        planner's bounds (R_i has degree <= D / i and coefficients below the
        bound of the lifted factors), call, grow on RS_ERR_CAPACITY, decode."""
        n = len(pairs)
        cw, fw = [], []
        for f, g in pairs:
            try:
                b = result_bound(f, g)
            except RsError:
                b = {"deg": 0, "limbs": 1, "bits": 0}
            D = max(b["deg"], 0)
            lh = (b["bits"] + D + int(math.ceil(0.5 * math.log2(D + 1))) + 2 + 31) // 32 + 1
            cw.append(max(1, b["limbs"]))
            fw.append([max(1, (D // m + 1) * lh) for m in range(1, max_mult + 1)])
        for _ in range(2):  # the second call has the exact sizes the first reported
            content = (rs_upoly * n)()
            facs = (rs_upoly * (n * max_mult))()
            cbuf = np.empty(sum(cw), dtype=np.uint32)
            fbuf = np.empty(sum(sum(w) for w in fw), dtype=np.uint32)
            base, co, fo = cbuf.ctypes.data, [], []
            off = 0
            for i in range(n):
                content[i].capacity_words = cw[i]
                content[i].coeffs = ctypes.cast(base + 4 * off, POINTER(c_uint32))
                co.append(off)
                off += cw[i]
            fbase, off = fbuf.ctypes.data, 0
            for i in range(n):
                for m in range(max_mult):
                    u = facs[i * max_mult + m]
                    u.capacity_words = fw[i][m]
                    u.coeffs = ctypes.cast(fbase + 4 * off, POINTER(c_uint32))
                    fo.append(off)
                    off += fw[i][m]
            nm = (c_int32 * n)()
            st = (c_int32 * n)()
            rc = call(content, facs, nm, st)
            grow = False
            for i in range(n):
                if st[i] != -2:
                    continue
                need_c = max(1, (content[i].deg + 1) * content[i].limbs)
                need_f = [max(1, (u.deg + 1) * u.limbs) for u in facs[i * max_mult:(i + 1) * max_mult]]
                if need_c > cw[i] or any(a > b for a, b in zip(need_f, fw[i])):
                    cw[i] = max(cw[i], need_c)
                    fw[i] = [max(a, b) for a, b in zip(need_f, fw[i])]
                    grow = True
            if not grow:
                break
        if raw:
            return list(st)
        msg = (self.lib.rs_last_error(self.h) or b"").decode() if rc < 0 else ""
        out = []
        for i in range(n):
            if st[i] != 0:
                out.append(RsError(st[i], msg if n == 1 else f"factorisation {i} failed"))
                continue
            c = limbs_to_ints(cbuf[co[i]:], content[i].deg, content[i].limbs)[0]
            r = []
            for m in range(max_mult):
                u = facs[i * max_mult + m]
                if u.deg > 0:
                    r.append((m + 1, limbs_to_ints(fbuf[fo[i * max_mult + m]:], u.deg, u.limbs)))
            out.append((c, r))
        return out

    def squarefree_info(self):
        """Stage times and counts of the last square-free call (dict)."""
        si = rs_sqf_info()
        _check(self.lib.rs_squarefree_info_get(self.h, ctypes.byref(si)), self.h)
        out = {k: getattr(si, k) for k, _ in rs_sqf_info._fields_ if k not in ("batch", "reserved")}
        out["batch"] = {k: getattr(si.batch, k) for k, _ in rs_batch_info._fields_ if k != "reserved"}
        return out

    def images(self, f, g, nprimes, npoints):
        """(primes[K], points[K, N], images[K, N]): images[k, i] =
        res(f(x, y), g(x, y), y) mod primes[k] at x = points[k, i]."""
        P = _Polys([f, g])
        primes = np.zeros(nprimes, dtype=np.uint32)
        pts = np.zeros((nprimes, npoints), dtype=np.uint32)
        imgs = np.zeros((nprimes, npoints), dtype=np.uint32)
        _check(self.lib.rs_images(self.h, ctypes.byref(P.structs[0]), ctypes.byref(P.structs[1]),
                                  nprimes, npoints, primes.ctypes.data_as(POINTER(c_uint32)),
                                  pts.ctypes.data_as(POINTER(c_uint32)),
                                  imgs.ctypes.data_as(POINTER(c_uint32))), self.h)
        return primes, pts, imgs

    def batch(self, pairs, stream=None):
        """A prepared batch; stream: a cudaStream_t handle (int) of this
        device to enqueue it on, None for the context's stream."""
        return Batch(self, pairs, stream)

    def autotune(self, pairs):
        """Tune the G1 launch for every workload class of these pairs that the
        process-wide cache lacks (nothing is computed)."""
        F, G = _Polys([p[0] for p in pairs]), _Polys([p[1] for p in pairs])
        _check(self.lib.rs_autotune(self.h, len(pairs), F.structs, G.structs), self.h)


def autotune_entries():
    """The tuner cache as a list of dicts (class, choice and timings)."""
    lib = load()
    n = c_int32()
    _check(lib.rs_autotune_entries(None, 0, ctypes.byref(n)))
    buf = (rs_tune_entry * max(n.value, 1))()
    _check(lib.rs_autotune_entries(buf, n.value, ctypes.byref(n)))
    return [{k: getattr(e, k) for k, _ in rs_tune_entry._fields_} for e in buf[: n.value]]


def autotune_save(path):
    _check(load().rs_autotune_save(os.fsencode(path)))


def autotune_load(path):
    _check(load().rs_autotune_load(os.fsencode(path)))


def autotune_clear():
    _check(load().rs_autotune_clear())


class Batch:
    """A prepared batch: inputs resident on the device, runs replayed."""

    def __init__(self, ctx, pairs, stream=None):
        self.ctx, self.lib, self.n = ctx, ctx.lib, len(pairs)
        self.F, self.G = _Polys([p[0] for p in pairs]), _Polys([p[1] for p in pairs])
        self.out = _Outputs(pairs)
        self.status = (c_int32 * max(self.n, 1))()
        h = c_void_p()
        _check(self.lib.rs_batch_create_on(ctx.h, self.n, self.F.structs, self.G.structs,
                                           c_void_p(stream) if stream else None, ctypes.byref(h)), ctx.h)
        self.h = h
        self.stream = stream or ctx.stream

    def upload(self, pairs=None):
        if pairs is not None:
            self.F, self.G = _Polys([p[0] for p in pairs]), _Polys([p[1] for p in pairs])
        _check(self.lib.rs_batch_upload(self.h, self.n, self.F.structs, self.G.structs), self.ctx.h)

    def run(self):
        _check(self.lib.rs_batch_run(self.h), self.ctx.h)

    def sync(self):
        _check(self.lib.rs_batch_sync(self.h), self.ctx.h)

    def results(self, raw=False):
        _check(self.lib.rs_batch_results(self.h, self.out.structs, self.status), self.ctx.h)
        return self.out.raw() if raw else self.out.ints()

    def info(self):
        i = rs_batch_info()
        _check(self.lib.rs_batch_info_get(self.h, ctypes.byref(i)), self.ctx.h)
        return {k: getattr(i, k) for k, _ in rs_batch_info._fields_}

    def close(self):
        if self.h and self.ctx.h:
            self.lib.rs_batch_destroy(self.h)
        self.h = None


class Server:
    """Continuous-batching request server of a context (rs_server_*)."""

    def __init__(self, ctx, max_inflight=0, max_batch=0, mem_limit_bytes=0):
        self.ctx, self.lib = ctx, ctx.lib
        _check(self.lib.rs_server_start(ctx.h, max_inflight, max_batch, mem_limit_bytes), ctx.h)

    def set_log(self, path):
        """Append one JSON line per finished request to path (None: stop)."""
        _check(self.lib.rs_server_set_log(self.ctx.h, os.fsencode(path) if path else None), self.ctx.h)

    def submit(self, f, g):
        P = _Polys([f, g])
        t = ctypes.c_uint64()
        _check(self.lib.rs_server_submit(self.ctx.h, ctypes.byref(P.structs[0]),
                                         ctypes.byref(P.structs[1]), ctypes.byref(t)), self.ctx.h)
        return t.value

    def _take(self, call, ticket, raw=False):
        """Run a poll/wait call with an empty buffer first; on RS_ERR_CAPACITY
        (ticket kept, size reported) allocate exactly and call again."""
        lat = c_double()
        out = rs_upoly()
        out.capacity_words = 0
        rc = call(out, lat)
        if rc == -2:
            words = max(1, (out.deg + 1) * out.limbs)
            buf = np.zeros(words, dtype=np.uint32)
            out.capacity_words = words
            out.coeffs = buf.ctypes.data_as(POINTER(c_uint32))
            rc = call(out, lat)
        else:
            buf = np.zeros(1, dtype=np.uint32)
        if rc in (RS_PENDING, -5):
            return None
        _check(rc, self.ctx.h)
        if raw:
            return (out.deg, out.limbs, buf), lat.value
        return limbs_to_ints(buf, out.deg, out.limbs), lat.value

    def poll(self, ticket, raw=False):
        """None while running, else (coefficients, latency_ms)."""
        return self._take(lambda o, l: self.lib.rs_server_poll(self.ctx.h, ticket, ctypes.byref(o),
                                                               ctypes.byref(l)), ticket, raw)

    def wait(self, ticket, timeout_us=-1, raw=False):
        """Block until done (or timeout: None); (coefficients, latency_ms)."""
        return self._take(lambda o, l: self.lib.rs_server_wait(self.ctx.h, ticket, ctypes.byref(o),
                                                               ctypes.byref(l), timeout_us),
                          ticket, raw)

    def stats(self):
        st = rs_server_stats()
        _check(self.lib.rs_server_stats_get(self.ctx.h, ctypes.byref(st)), self.ctx.h)
        return {k: getattr(st, k) for k, _ in rs_server_stats._fields_}

    def stop(self):
        _check(self.lib.rs_server_stop(self.ctx.h), self.ctx.h)
