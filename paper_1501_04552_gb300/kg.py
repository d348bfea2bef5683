"""Thin ctypes binding of libkg.so (C ABI declared in include/kg.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Importing this module loads the library and raises ImportError when it
has not been built (``python -c "import __graft_entry__ as g; g.build()"``); there
is no fallback.  Host arrays are numpy float64 arrays [z][y][x]; device buffers may
be passed as torch CUDA tensors or raw integer pointers.
"""
import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "kg.h")

KG_OK = 0
KG_EINVAL = -1
KG_ENOTSUP = -2
KG_ENOMEM = -3
KG_ECUDA = -4
KG_ETIMEOUT = -5
KG_EDRIFT = -6
KG_ENOTIMPL = -7
KG_ESTATE = -8

KG_FP64 = 0
KG_DF64 = 1
KG_MIXED = 2

KG_SCHEME_EQ2 = 0
KG_SCHEME_COMPOSED4 = 1
SCHEMES = {"eq2": KG_SCHEME_EQ2, "composed4": KG_SCHEME_COMPOSED4}
PRECISIONS = {"fp64": KG_FP64, "df64": KG_DF64, "mixed": KG_MIXED}


class kg_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("energy_every", C.c_int), ("nonlinearity", C.c_double),
                ("blowup_threshold", C.c_double), ("drift_tol", C.c_double), ("tune_cache", C.c_char_p)]


class kg_mlp_cfg(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("T", C.c_double),
                ("seed", C.c_ulonglong)]


class KgError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with status %d: %s" % (what, code, last_error()))
        self.code = code


if not os.path.exists(LIB_PATH):
    raise ImportError("libkg.so is not built (run paper_1501_04552_gb300/build.py); no CPU fallback exists")

lib = C.CDLL(LIB_PATH)
_vp = C.c_void_p
_sig = {
    "kg_init": ([C.c_int, C.c_double, C.c_double, _vp, _vp], C.c_int),
    "kg_init_device": ([C.c_int, C.c_double, C.c_double, _vp, _vp], C.c_int),
    "kg_step": ([C.c_int], C.c_int),
    "kg_energy": ([C.POINTER(C.c_double)], C.c_int),
    "kg_fetch": ([_vp], C.c_int),
    "kg_fetch_device": ([_vp], C.c_int),
    "kg_finalize": ([], C.c_int),
    "kg_set_stream": ([_vp], C.c_int),
    "kg_set_options": ([C.POINTER(kg_options)], C.c_int),
    "kg_get_options": ([C.POINTER(kg_options)], C.c_int),
    "kg_set_scheme": ([C.c_int], C.c_int),
    "kg_get_scheme": ([C.POINTER(C.c_int)], C.c_int),
    "kg_set_xy_fusion": ([C.c_int], C.c_int),
    "kg_get_xy_fusion": ([C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "kg_status": ([C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_double)],
                  C.c_int),
    "kg_fetch_spectral": ([_vp, _vp], C.c_int),
    "kg_step_timed": ([C.c_int, C.POINTER(C.c_float)], C.c_int),
    "kg_memory": ([C.POINTER(C.c_size_t)], C.c_int),
    "kg_init_complex": ([C.c_int, C.c_double, C.c_double, _vp, _vp], C.c_int),
    "kg_init_complex_device": ([C.c_int, C.c_double, C.c_double, _vp, _vp], C.c_int),
    "kg_fetch_complex": ([_vp], C.c_int),
    "kg_fetch_complex_device": ([_vp], C.c_int),
    "kg_save_state": ([_vp, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
    "kg_load_state": ([_vp, C.c_size_t], C.c_int),
    "kg_state_checksum": ([_vp, C.c_size_t], C.c_ulonglong),
    "kg_last_error": ([], C.c_char_p),
    "kg_energy_q_noalloc": ([C.c_int, C.c_double, C.c_double, _vp, _vp, _vp, _vp], C.c_int),
    "kg_ens_init": ([C.c_int, _vp, C.c_double, C.c_double, _vp, _vp], C.c_int),
    "kg_ens_run": ([C.c_int, C.c_double, C.POINTER(C.c_longlong), C.POINTER(C.c_double)], C.c_int),
    "kg_ens_results": ([_vp, _vp, _vp, _vp], C.c_int),
    "kg_ens_features": ([_vp], C.c_int),
    "kg_ens_fetch": ([C.c_int, _vp], C.c_int),
    "kg_ens_tune": ([C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "kg_ens_schedule": ([C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "kg_ens_set_schedule": ([C.c_int, C.c_int, C.c_int], C.c_int),
    "kg_ens_set_tune_cache": ([C.c_char_p], C.c_int),
    "kg_ens_finalize": ([], C.c_int),
    "kg_gaussian_features": ([C.c_int, C.c_int, C.c_double, _vp, _vp, _vp], C.c_int),
    "kg_mlp_param_count": ([], C.c_int),
    "kg_mlp_set_params": ([_vp], C.c_int),
    "kg_mlp_get_params": ([_vp], C.c_int),
    "kg_mlp_grad": ([_vp, _vp, _vp, C.c_int, C.c_double, _vp, C.POINTER(C.c_double)], C.c_int),
    "kg_mlp_adam_step": ([_vp, C.c_double], C.c_int),
    "kg_mlp_train": ([_vp, _vp, _vp, C.c_int, C.POINTER(kg_mlp_cfg), C.POINTER(C.c_double)], C.c_int),
    "kg_mlp_predict": ([_vp, C.c_int, _vp, _vp], C.c_int),
    "kg_mlp_finalize": ([], C.c_int),
}
_state = {"N": None}
for _name, (_args, _res) in _sig.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def header_symbols(path=HEADER):
    """names of the entry points declared in include/kg.h"""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kg_[a-z_0-9]+)\s*\(", text)))


def last_error():
    s = lib.kg_last_error()
    return s.decode() if s else ""


def _check(rc, what, ok=(KG_OK,)):
    if rc not in ok:
        raise KgError(rc, what)
    return rc


def _host(a, n3, name):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n3:
        raise ValueError("%s must hold N^3 = %d values" % (name, n3))
    return a


def _dptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def kg_init(N, L, dt, u0, v0=None):
    u = _host(u0, N ** 3, "u0")
    v = None if v0 is None else _host(v0, N ** 3, "v0")
    _check(lib.kg_init(N, L, dt, u.ctypes.data, None if v is None else v.ctypes.data), "kg_init")
    _state["N"] = N
    _state["cplx"] = False


def kg_init_device(N, L, dt, d_u0, d_v0=None):
    _check(lib.kg_init_device(N, L, dt, _dptr(d_u0), _dptr(d_v0)), "kg_init_device")
    _state["N"] = N
    _state["cplx"] = False


def _host_c(a, n3, name):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.size != n3:
        raise ValueError("%s must hold N^3 = %d complex values" % (name, n3))
    return a


def kg_init_complex(N, L, dt, u0, v0=None):
    """complex field: u0, v0 are N^3 complex arrays ([z][y][x]); v0 may be None (= 0)"""
    u = _host_c(u0, N ** 3, "u0")
    v = None if v0 is None else _host_c(v0, N ** 3, "v0")
    _check(lib.kg_init_complex(N, L, dt, u.ctypes.data, None if v is None else v.ctypes.data), "kg_init_complex")
    _state["N"] = N
    _state["cplx"] = True


def kg_init_complex_device(N, L, dt, d_u0, d_v0=None):
    """device pointers (or complex128 torch tensors) of N^3 complex values each"""
    _check(lib.kg_init_complex_device(N, L, dt, _dptr(d_u0), _dptr(d_v0)), "kg_init_complex_device")
    _state["N"] = N
    _state["cplx"] = True


def kg_fetch_complex(N=None, out=None):
    if out is None:
        N = N or _state["N"]
        out = np.empty((N, N, N), dtype=np.complex128)
    _check(lib.kg_fetch_complex(out.ctypes.data), "kg_fetch_complex")
    return out


def kg_fetch_complex_device(d_u):
    _check(lib.kg_fetch_complex_device(_dptr(d_u)), "kg_fetch_complex_device")


def kg_step(n=1):
    _check(lib.kg_step(int(n)), "kg_step")


def kg_energy(allow_drift=False):
    E = C.c_double()
    rc = lib.kg_energy(C.byref(E))
    _check(rc, "kg_energy", ok=(KG_OK, KG_EDRIFT) if allow_drift else (KG_OK,))
    return E.value


def kg_fetch(N=None, out=None):
    if out is None:
        N = N or _state["N"]
        out = np.empty((N, N, N), dtype=np.float64)
    _check(lib.kg_fetch(out.ctypes.data), "kg_fetch")
    return out


def kg_fetch_device(d_u):
    _check(lib.kg_fetch_device(_dptr(d_u)), "kg_fetch_device")


def kg_finalize():
    _check(lib.kg_finalize(), "kg_finalize")


def kg_set_stream(stream):
    ptr = stream if (stream is None or isinstance(stream, int)) else stream.cuda_stream
    _check(lib.kg_set_stream(ptr), "kg_set_stream")


def kg_set_options(precision=KG_DF64, energy_every=0, nonlinearity=1.0, blowup_threshold=0.0, drift_tol=0.0,
                   tune_cache=None):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    path = None if tune_cache is None else os.fsencode(tune_cache)
    o = kg_options(int(precision), int(energy_every), float(nonlinearity), float(blowup_threshold), float(drift_tol),
                   path)
    _check(lib.kg_set_options(C.byref(o)), "kg_set_options")


def kg_get_options():
    o = kg_options()
    _check(lib.kg_get_options(C.byref(o)), "kg_get_options")
    d = {f: getattr(o, f) for f, _ in kg_options._fields_}
    d["tune_cache"] = None if d["tune_cache"] is None else os.fsdecode(d["tune_cache"])
    return d


def kg_set_scheme(scheme=KG_SCHEME_EQ2):
    """time-stepping scheme of the next kg_init: "eq2" (Eq. (2)) or "composed4" (fourth order)"""
    if isinstance(scheme, str):
        scheme = SCHEMES[scheme]
    _check(lib.kg_set_scheme(int(scheme)), "kg_set_scheme")


def kg_get_scheme():
    v = C.c_int()
    _check(lib.kg_get_scheme(C.byref(v)), "kg_get_scheme")
    return v.value


def kg_set_xy_fusion(on=True):
    """the cluster-fused inverse-y / x / forward-y pass for the FP32 passes (next kg_step)"""
    _check(lib.kg_set_xy_fusion(1 if on else 0), "kg_set_xy_fusion")


def kg_get_xy_fusion():
    """(as set, used by the current context)"""
    on, active = C.c_int(), C.c_int()
    _check(lib.kg_get_xy_fusion(C.byref(on), C.byref(active)), "kg_get_xy_fusion")
    return bool(on.value), bool(active.value)


def kg_status():
    lvl, fr, bl, mx = C.c_longlong(), C.c_int(), C.c_longlong(), C.c_double()
    _check(lib.kg_status(C.byref(lvl), C.byref(fr), C.byref(bl), C.byref(mx)), "kg_status")
    return {"level": lvl.value, "frozen": bool(fr.value), "blowup_level": bl.value, "maxabs": mx.value}


def kg_fetch_spectral(N):
    a = np.empty((N, N, N if _state.get("cplx") else N // 2 + 1), dtype=np.complex128)
    b = np.empty_like(a)
    _check(lib.kg_fetch_spectral(a.ctypes.data, b.ctypes.data), "kg_fetch_spectral")
    return a, b


# slots of kg_step_timed: the z pass is one kernel, so "z" holds all of it and the
# "update" and "zi" slots read 0
STEP_KERNELS = ["x", "yf", "z", "update", "zi", "yi"]


def kg_step_timed(n):
    """summed device ms of the kernel groups of a step (slot names in STEP_KERNELS)"""
    ms = (C.c_float * 6)()
    _check(lib.kg_step_timed(int(n), ms), "kg_step_timed")
    return [ms[i] for i in range(6)]


def kg_memory():
    b = C.c_size_t()
    _check(lib.kg_memory(C.byref(b)), "kg_memory")
    return b.value


class kg_state_header(C.Structure):
    """mirror of kg_state_header in include/kg.h (256 bytes, machine byte order)"""
    _fields_ = [("magic", C.c_char * 8), ("version", C.c_uint), ("header_bytes", C.c_uint),
                ("N", C.c_int), ("precision", C.c_int), ("energy_every", C.c_int), ("frozen", C.c_int),
                ("L", C.c_double), ("dt", C.c_double), ("nonlinearity", C.c_double),
                ("blowup_threshold", C.c_double), ("drift_tol", C.c_double),
                ("level", C.c_longlong), ("blowup_level", C.c_longlong), ("maxabs_last", C.c_double),
                ("P_last", C.c_double), ("P_last_level", C.c_longlong), ("Q_last", C.c_double),
                ("Q_last_level", C.c_longlong), ("have_E0", C.c_int), ("pad0", C.c_int), ("E0", C.c_double),
                ("payload_bytes", C.c_ulonglong), ("checksum", C.c_ulonglong), ("complex_field", C.c_int),
                ("scheme", C.c_int), ("reserved", C.c_ubyte * 88)]


STATE_HEADER_BYTES = 256
KG_STATE_MAGIC = b"KGSTATE1"
KG_STATE_VERSION = 1


def state_header(buf):
    """the kg_state_header at the start of a checkpoint buffer"""
    return kg_state_header.from_buffer_copy(np.ascontiguousarray(buf[:STATE_HEADER_BYTES]).tobytes())


def kg_save_state():
    """the context as one checkpoint buffer (numpy uint8: 256-byte header, then the state)"""
    need = C.c_size_t(0)
    _check(lib.kg_save_state(None, 0, C.byref(need)), "kg_save_state")
    buf = np.empty(need.value, dtype=np.uint8)
    _check(lib.kg_save_state(buf.ctypes.data, buf.size, C.byref(need)), "kg_save_state")
    return buf


def kg_load_state(buf):
    """replace the context by a checkpoint written by kg_save_state"""
    b = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if not isinstance(buf, np.ndarray) else buf)
    if b.dtype != np.uint8:
        b = b.view(np.uint8)
    _check(lib.kg_load_state(b.ctypes.data, b.size), "kg_load_state")
    h = state_header(b)
    _state["N"] = h.N
    _state["cplx"] = bool(h.complex_field)


def kg_state_checksum(payload):
    b = np.ascontiguousarray(payload).view(np.uint8)
    return int(lib.kg_state_checksum(b.ctypes.data, b.size))


def kg_last_error():
    return last_error()


# ---------------------------------------------------------------------------
# batched ensemble
# ---------------------------------------------------------------------------
_ens = {"Ns": None}


def kg_ens_init(Ns, L, dt, A, s):
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    A = np.ascontiguousarray(A, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    if not (Ns.size == A.size == s.size):
        raise ValueError("Ns, A and s must have one entry per instance")
    _check(lib.kg_ens_init(Ns.size, Ns.ctypes.data, L, dt, A.ctypes.data, s.ctypes.data), "kg_ens_init")
    _ens["Ns"] = Ns.copy()


def kg_ens_run(max_steps, threshold=0.0):
    done, ms = C.c_longlong(), C.c_double()
    _check(lib.kg_ens_run(int(max_steps), float(threshold), C.byref(done), C.byref(ms)), "kg_ens_run")
    return done.value, ms.value


def kg_ens_results():
    n = _ens["Ns"].size
    fr = np.empty(n, dtype=np.int32)
    bl = np.empty(n, dtype=np.int64)
    lv = np.empty(n, dtype=np.int64)
    mx = np.empty(n, dtype=np.float64)
    _check(lib.kg_ens_results(fr.ctypes.data, bl.ctypes.data, lv.ctypes.data, mx.ctypes.data), "kg_ens_results")
    return {"frozen": fr.astype(bool), "blowup_level": bl, "level": lv, "maxabs": mx}


def kg_ens_features():
    out = np.empty((_ens["Ns"].size, 4), dtype=np.float64)
    _check(lib.kg_ens_features(out.ctypes.data), "kg_ens_features")
    return out


def kg_ens_fetch(i):
    N = int(_ens["Ns"][i])
    out = np.empty((N, N, N), dtype=np.float64)
    _check(lib.kg_ens_fetch(int(i), out.ctypes.data), "kg_ens_fetch")
    return out


def kg_ens_tune(steps=3):
    b, o = C.c_int(), C.c_int()
    _check(lib.kg_ens_tune(int(steps), C.byref(b), C.byref(o)), "kg_ens_tune")
    return b.value, o.value


def kg_ens_schedule():
    """(schedule, CTAs per SM, unit order) of the current ensemble"""
    sc, b, o = C.c_int(), C.c_int(), C.c_int()
    _check(lib.kg_ens_schedule(C.byref(sc), C.byref(b), C.byref(o)), "kg_ens_schedule")
    return sc.value, b.value, o.value


def kg_ens_set_schedule(sched, blocks_per_sm, order):
    _check(lib.kg_ens_set_schedule(int(sched), int(blocks_per_sm), int(order)), "kg_ens_set_schedule")


def kg_ens_set_tune_cache(path):
    _check(lib.kg_ens_set_tune_cache(None if path is None else os.fsencode(path)), "kg_ens_set_tune_cache")


def kg_ens_finalize():
    _check(lib.kg_ens_finalize(), "kg_ens_finalize")


def kg_gaussian_features(N, L, A, s):
    A = np.ascontiguousarray(A, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.empty((A.size, 4), dtype=np.float64)
    _check(lib.kg_gaussian_features(A.size, int(N), float(L), A.ctypes.data, s.ctypes.data, out.ctypes.data),
           "kg_gaussian_features")
    return out


# ---------------------------------------------------------------------------
# blow-up ranker network
# ---------------------------------------------------------------------------
def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


def kg_mlp_param_count():
    return lib.kg_mlp_param_count()


def kg_mlp_set_params(params):
    p = _f32(params)
    if p.size != kg_mlp_param_count():
        raise ValueError("parameter vector must hold %d values" % kg_mlp_param_count())
    _check(lib.kg_mlp_set_params(p.ctypes.data), "kg_mlp_set_params")


def kg_mlp_get_params():
    out = np.empty(kg_mlp_param_count(), dtype=np.float32)
    _check(lib.kg_mlp_get_params(out.ctypes.data), "kg_mlp_get_params")
    return out


def kg_mlp_grad(X, y, logt, T=10.0):
    X, y, logt = _f32(X), _f32(y), _f32(logt)
    g = np.empty(kg_mlp_param_count(), dtype=np.float32)
    loss = C.c_double()
    _check(lib.kg_mlp_grad(X.ctypes.data, y.ctypes.data, logt.ctypes.data, X.shape[0], T, g.ctypes.data,
                           C.byref(loss)), "kg_mlp_grad")
    return loss.value, g


def kg_mlp_adam_step(grad, lr=1e-3):
    g = _f32(grad)
    _check(lib.kg_mlp_adam_step(g.ctypes.data, lr), "kg_mlp_adam_step")


def kg_mlp_train(X, y, logt, epochs=100, batch=256, lr=1e-3, T=10.0, seed=1):
    X, y, logt = _f32(X), _f32(y), _f32(logt)
    cfg = kg_mlp_cfg(int(epochs), int(batch), float(lr), float(T), int(seed))
    loss = C.c_double()
    _check(lib.kg_mlp_train(X.ctypes.data, y.ctypes.data, logt.ctypes.data, X.shape[0], C.byref(cfg),
                            C.byref(loss)), "kg_mlp_train")
    return loss.value


def kg_mlp_predict(X):
    X = _f32(X)
    n = X.shape[0]
    p = np.empty(n, dtype=np.float32)
    t = np.empty(n, dtype=np.float32)
    _check(lib.kg_mlp_predict(X.ctypes.data, n, p.ctypes.data, t.ctypes.data), "kg_mlp_predict")
    return p, t


def kg_mlp_finalize():
    _check(lib.kg_mlp_finalize(), "kg_mlp_finalize")

