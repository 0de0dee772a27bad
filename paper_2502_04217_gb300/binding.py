"""Thin ctypes binding of libsdft_ipm.so (include/sdft_ipm.h), same names as the C ABI.

Only argument marshalling lives here: every step of the solve runs in the
CUDA library.  Loading fails loudly when the library has not been built;
there is no fallback.

Arrays may be torch tensors (CPU or CUDA), numpy arrays, or raw integer
addresses.  The C functions documented as taking device pointers must be
given CUDA tensors (or device addresses).
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsdft_ipm.so")

IPM_OK, IPM_ERR_ARG, IPM_ERR_CUDA, IPM_ERR_OOM, IPM_MAXITER, IPM_KRYLOV_MAXITER, IPM_NUMERICAL, IPM_TIMEOUT = range(8)
IPM_FP64, IPM_MIXED = 0, 1
STATUS_NAMES = {0: "IPM_OK", 1: "IPM_ERR_ARG", 2: "IPM_ERR_CUDA", 3: "IPM_ERR_OOM", 4: "IPM_MAXITER",
                5: "IPM_KRYLOV_MAXITER", 6: "IPM_NUMERICAL", 7: "IPM_TIMEOUT"}
PROFILE_CLASSES = {"fft_row": 0, "fft_col": 1, "fft_middle": 2, "pcg_update": 3, "ipm_other": 4, "prepare": 6,
                   "step": 7, "certificate": 8}


class ipm_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("gap_tol", ctypes.c_double), ("cg_tol", ctypes.c_double),
                ("cg_relative", ctypes.c_int), ("max_ipm", ctypes.c_int), ("max_cg", ctypes.c_int),
                ("sigma", ctypes.c_double), ("sigma_slow", ctypes.c_double), ("tau", ctypes.c_double),
                ("lambda_relative", ctypes.c_int), ("cg_chunk", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("autotune", ctypes.c_int), ("tile_e", ctypes.c_int), ("tile_p", ctypes.c_int),
                ("refine_every", ctypes.c_int), ("tile_engine", ctypes.c_int),
                ("sigma_rule", ctypes.c_int), ("sigma_min", ctypes.c_double), ("exact_residual", ctypes.c_int),
                ("precond_rho", ctypes.c_double), ("pdl", ctypes.c_int),
                ("krylov", ctypes.c_int), ("tile_kstage", ctypes.c_int)]


class ipm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("ipm_iters", ctypes.c_int), ("cg_iters_total", ctypes.c_int),
                ("cg_iters_max", ctypes.c_int), ("primal", ctypes.c_double), ("dual", ctypes.c_double),
                ("rel_gap", ctypes.c_double), ("mu", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("seconds", ctypes.c_double), ("kkt_products", ctypes.c_int),
                ("refinements", ctypes.c_int), ("exact_products", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class IpmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_P = ctypes.c_void_p
_SIGNATURES = {
    "ipm_default_options": (None, [ctypes.POINTER(ipm_options)]),
    "ipm_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int64), _P, _P,
                                  ctypes.c_double, ctypes.POINTER(ipm_options), _P]),
    "ipm_set_problem": (ctypes.c_int, [_P, _P, _P, ctypes.c_double]),
    "ipm_set_options": (ctypes.c_int, [_P, ctypes.POINTER(ipm_options)]),
    "ipm_solve": (ctypes.c_int, [_P, ctypes.POINTER(ipm_result)]),
    "ipm_sizes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "gapply": (ctypes.c_int, [_P, _P, _P]),
    "kkt_apply": (ctypes.c_int, [_P, _P, _P]),
    "ipm_test_stage_stall": (ctypes.c_int, [_P, ctypes.c_int]),
    "precond_apply": (ctypes.c_int, [_P, _P, _P]),
    "ipm_set_sigma": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ipm_set_point": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "ipm_get_point": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "ipm_get_spectrum": (ctypes.c_int, [_P, _P]),
    "ipm_pack_beta": (ctypes.c_int, [_P, _P, _P]),
    "ipm_unpack_beta": (ctypes.c_int, [_P, _P, _P]),
    "ipm_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "ipm_profile_get": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double)]),
    "ipm_create_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ipm_options), _P]),
    "ipm_solve_batch": (ctypes.c_int, [_P, ctypes.POINTER(ipm_result)]),
    "ipm_batch_size": (ctypes.c_int, [_P]),
    "ipm_batch_member": (_P, [_P, ctypes.c_int]),
    "ipm_batch_last_error": (ctypes.c_char_p, [_P]),
    "ipm_destroy_batch": (None, [_P]),
    "ws_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_uint64, _P]),
    "ws_destroy": (None, [_P]),
    "ws_num_params": (ctypes.c_int64, [_P]),
    "ws_get_params": (ctypes.c_int, [_P, _P]),
    "ws_set_params": (ctypes.c_int, [_P, _P]),
    "ws_get_grads": (ctypes.c_int, [_P, _P]),
    "ws_forward": (ctypes.c_int, [_P, _P, _P]),
    "ws_predict": (ctypes.c_int, [_P, _P, ctypes.c_double]),
    "ws_train_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]),
    "ws_conv_forward": (ctypes.c_int, [ctypes.c_int] * 5 + [_P, _P, _P, ctypes.c_int, _P, _P, _P]),
    "ws_test_conv_stall": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "ws_conv_wgrad": (ctypes.c_int, [ctypes.c_int] * 6 + [_P, _P, _P, _P, _P]),
    "gapply_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), _P, _P, _P, _P]),
    "ipm_describe": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.c_int]),
    "ipm_last_error": (ctypes.c_char_p, [_P]),
    "ipm_destroy": (None, [_P]),
}

_lib = None


def load(path=None):
    """Load libsdft_ipm.so (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def addr(x):
    """Address of an array-like: torch tensor, numpy array or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def default_options(**kw):
    o = ipm_options()
    load().ipm_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _check(status, handle=None):
    if status != IPM_OK:
        msg = load().ipm_last_error(handle)
        raise IpmError(status, msg.decode() if msg else "")
    return status


# ---- functions with the C names ---------------------------------------------------------

def ipm_create(dims, mask, y, lam, options=None, stream=None):
    """Returns a handle (int).  mask: uint8, y: float64, host or device, n elements each."""
    lib = load()
    h = _P()
    d = (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])
    st = lib.ipm_create(ctypes.byref(h), len(dims), d, addr(mask), addr(y), float(lam),
                        ctypes.byref(options) if options is not None else None, stream)
    _check(st, None)
    return h.value


def ipm_set_problem(h, mask, y, lam):
    return _check(load().ipm_set_problem(h, addr(mask), addr(y), float(lam)), h)


def ipm_set_options(h, options):
    return _check(load().ipm_set_options(h, ctypes.byref(options)), h)


def ipm_solve(h, check=True):
    r = ipm_result()
    st = load().ipm_solve(h, ctypes.byref(r))
    if check and st not in (IPM_OK, IPM_KRYLOV_MAXITER):
        _check(st, h)
    out = r.as_dict()
    out["lambda"] = out.pop("lambda_")
    out["status_name"] = STATUS_NAMES.get(st, st)
    return out


def ipm_sizes(h):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().ipm_sizes(h, ctypes.byref(a), ctypes.byref(b)), h)
    return a.value, b.value


def gapply(h, p, q):
    return _check(load().gapply(h, addr(p), addr(q)), h)


def kkt_apply(h, p, q):
    return _check(load().kkt_apply(h, addr(p), addr(q)), h)


def ipm_test_stage_stall(h, wait_log2):
    """Failure-detection test hook: the next kkt_apply on h drops one staged operand copy."""
    return _check(load().ipm_test_stage_stall(h, int(wait_log2)), h)


def precond_apply(h, r, z):
    return _check(load().precond_apply(h, addr(r), addr(z)), h)


def ipm_set_sigma(h, s1, nu1, s2, nu2):
    return _check(load().ipm_set_sigma(h, addr(s1), addr(nu1), addr(s2), addr(nu2)), h)


def ipm_set_point(h, w):
    arr = (_P * 6)(*[addr(v) for v in w])
    return _check(load().ipm_set_point(h, arr), h)


def ipm_get_point(h, w):
    arr = (_P * 6)(*[addr(v) for v in w])
    return _check(load().ipm_get_point(h, arr), h)


def ipm_get_spectrum(h, v_half):
    return _check(load().ipm_get_spectrum(h, addr(v_half)), h)


def ipm_pack_beta(h, v_half, beta):
    return _check(load().ipm_pack_beta(h, addr(v_half), addr(beta)), h)


def ipm_unpack_beta(h, beta, v_half):
    return _check(load().ipm_unpack_beta(h, addr(beta), addr(v_half)), h)


def ipm_profile_enable(h, on=True):
    return _check(load().ipm_profile_enable(h, 1 if on else 0), h)


def ipm_profile_get(h, k):
    n, ms = ctypes.c_int64(), ctypes.c_double()
    _check(load().ipm_profile_get(h, int(k), ctypes.byref(n), ctypes.byref(ms)), h)
    return n.value, ms.value


def ipm_create_batch(problems, options=None, stream=None):
    """problems: list of (dims, mask, y, lam).  Returns a batch handle (int)."""
    lib = load()
    count = len(problems)
    nd = (ctypes.c_int * count)(*[len(p[0]) for p in problems])
    flat = []
    for p in problems:
        flat += [int(v) for v in p[0]] + [0] * (3 - len(p[0]))
    dims = (ctypes.c_int64 * (3 * count))(*flat)
    masks = (_P * count)(*[addr(p[1]) for p in problems])
    ys = (_P * count)(*[addr(p[2]) for p in problems])
    lams = (ctypes.c_double * count)(*[float(p[3]) for p in problems])
    b = _P()
    st = lib.ipm_create_batch(ctypes.byref(b), count, nd, dims, masks, ys, lams,
                              ctypes.byref(options) if options is not None else None, stream)
    _check(st, None)
    return b.value


def ipm_solve_batch(b, check=True):
    lib = load()
    count = lib.ipm_batch_size(b)
    res = (ipm_result * count)()
    st = lib.ipm_solve_batch(b, res)
    if check and st not in (IPM_OK, IPM_KRYLOV_MAXITER):
        m = lib.ipm_batch_last_error(b)
        raise IpmError(st, m.decode() if m else "")
    out = []
    for r in res:
        d = r.as_dict()
        d["lambda"] = d.pop("lambda_")
        out.append(d)
    return out


def ipm_batch_member(b, i):
    return load().ipm_batch_member(b, int(i))


def ipm_destroy_batch(b):
    load().ipm_destroy_batch(b)


def ws_create(seed=0, stream=None):
    n = _P()
    _check(load().ws_create(ctypes.byref(n), int(seed), stream), None)
    return n.value


def ws_destroy(n):
    load().ws_destroy(n)


def ws_num_params(n):
    return int(load().ws_num_params(n))


def ws_get_params(n, dst):
    return _check(load().ws_get_params(n, addr(dst)), None)


def ws_set_params(n, src):
    return _check(load().ws_set_params(n, addr(src)), None)


def ws_get_grads(n, dst):
    return _check(load().ws_get_grads(n, addr(dst)), None)


def ws_forward(n, h, y=None):
    return _check(load().ws_forward(n, h, addr(y)), None)


def ws_predict(n, h, mu_scale=1e-3):
    return _check(load().ws_predict(n, h, float(mu_scale)), None)


def ws_train_step(n, h, beta_star, lr):
    loss = ctypes.c_double()
    _check(load().ws_train_step(n, h, addr(beta_star), float(lr), ctypes.byref(loss)), None)
    return loss.value


def ws_conv_forward(cin, cout, dims, x, w, bias, relu, aux, y, stream=None):
    return _check(load().ws_conv_forward(cin, cout, *[int(d) for d in dims], addr(x), addr(w), addr(bias),
                                         int(relu), addr(aux), addr(y), stream), None)


def ws_test_conv_stall(drop_triple, wait_log2):
    """Failure-detection test hook: the next tensor-core convolution drops one copy."""
    return _check(load().ws_test_conv_stall(int(drop_triple), int(wait_log2)), None)


def ws_conv_wgrad(cin, m, mout, dims, x, dy, dw, db, stream=None):
    return _check(load().ws_conv_wgrad(cin, m, mout, *[int(d) for d in dims], addr(x), addr(dy), addr(dw),
                                       addr(db), stream), None)


def gapply_noalloc(dims, mask, p, q, stream=None):
    """Handle-free, allocation-free q = M_perp^T M_perp p (device mask, p, q)."""
    d = (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])
    return _check(load().gapply_noalloc(len(dims), d, addr(mask), addr(p), addr(q), stream), None)


def ipm_describe(h):
    """The FFT tile plan of the handle (dict)."""
    import json
    buf = ctypes.create_string_buffer(4096)
    load().ipm_describe(h, buf, 4096)
    return json.loads(buf.value.decode())


def ipm_last_error(h=None):
    m = load().ipm_last_error(h)
    return m.decode() if m else ""


def ipm_destroy(h):
    load().ipm_destroy(h)
