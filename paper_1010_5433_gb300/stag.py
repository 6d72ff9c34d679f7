"""ctypes binding of libstag (include/stag.h).  Argument marshalling only: every
step of the computation runs in the CUDA library; this module converts
Python values and torch tensors into the plain pointers and structs of the C
ABI.  There is no CPU fallback: if the compiled library is missing, loading
fails with an error.

Functions keep the C names (stag_create, stag_dslash, ...).  Tensor arguments
are torch CUDA tensors in the layouts the header documents; raw integer
device pointers are accepted as well.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libstag.so")

STAG_FP64, STAG_FP32, STAG_FP32_12, STAG_BF16_12 = 0, 1, 2, 3
STAG_ACTION_UNIMPROVED, STAG_ACTION_ASQTAD = 0, 1
STAG_MAX_SHIFTS = 32
STAG_MAX_FLAVOURS = 2
STATUS = {0: "ok", 1: "invalid argument", 2: "allocation failed", 3: "CUDA error",
          4: "solver did not converge", 5: "device wait timed out", 6: "NaN or Inf", 7: "no gauge field"}


class StagError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {detail}".strip())


class stag_lattice(C.Structure):
    _fields_ = [("dims", C.c_int * 4), ("t_antiperiodic", C.c_int), ("cuda_stream", C.c_void_p)]


class stag_rational(C.Structure):
    _fields_ = [("n", C.c_int), ("a0", C.c_double), ("alpha", C.POINTER(C.c_double)),
                ("beta", C.POINTER(C.c_double))]


class stag_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("shift_iterations", C.c_int * STAG_MAX_SHIFTS),
                ("true_residual", C.c_double * STAG_MAX_SHIFTS), ("reliable_updates", C.c_int)]


class stag_flavour(C.Structure):
    _fields_ = [("mass", C.c_double), ("n_pf", C.c_int), ("level", C.c_int), ("hb", stag_rational),
                ("md", stag_rational), ("met", stag_rational)]


class stag_hmc(C.Structure):
    _fields_ = [("beta", C.c_double), ("tau", C.c_double), ("n_outer", C.c_int), ("n_gauge", C.c_int),
                ("n_flavours", C.c_int), ("flavour", stag_flavour * STAG_MAX_FLAVOURS),
                ("tol_md", C.c_double), ("tol_met", C.c_double), ("max_iter", C.c_int),
                ("md_prec", C.c_int), ("seed", C.c_ulonglong), ("counter", C.c_ulonglong),
                ("ext_mom", C.c_void_p), ("ext_xi", C.c_void_p), ("ext_phi", C.c_void_p), ("ext_uniform", C.c_double),
                ("no_metropolis", C.c_int), ("flip_momenta", C.c_int), ("use_surrogate", C.c_int),
                ("n_mid", C.c_int)]


class stag_kernel_profile(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("sampled", C.c_int), ("sampled_ms", C.c_double),
                ("bytes_per_launch", C.c_double)]


class stag_traj(C.Structure):
    _fields_ = [("dH", C.c_double), ("H0", C.c_double), ("H1", C.c_double), ("plaq", C.c_double),
                ("accepted", C.c_int), ("cg_iterations", C.c_longlong), ("reliable_updates", C.c_int),
                ("seconds", C.c_double), ("t_heatbath", C.c_double), ("t_fermion", C.c_double),
                ("t_gauge", C.c_double), ("t_metropolis", C.c_double)]


# ctypes signature of every function include/stag.h declares: (argument
# types, result type)
_vp, _i, _d = C.c_void_p, C.c_int, C.c_double
SIGNATURES = {
    "stag_create": ([C.POINTER(stag_lattice), C.POINTER(_vp)], _i),
    "stag_destroy": ([_vp], None),
    "stag_strerror": ([_i], C.c_char_p),
    "stag_last_cuda_error": ([_vp], C.c_char_p),
    "stag_set_stream": ([_vp, _vp], _i),
    "stag_device_bytes": ([_vp], C.c_size_t),
    "stag_abi_sizeof": ([_i], C.c_size_t),
    "stag_load_gauge": ([_vp, _vp], _i),
    "stag_load_gauge_device": ([_vp, _vp], _i),
    "stag_store_gauge": ([_vp, _vp], _i),
    "stag_dslash": ([_vp, _i, _i, _i, _vp, _vp], _i),
    "stag_apply_a": ([_vp, _d, _d, _i, _i, _vp, _vp], _i),
    "stag_apply_a_noalloc": ([_vp, _d, _d, _i, _i, _vp, _vp], _i),
    "stag_set_action": ([_vp, _i, _d], _i),
    "stag_asqtad_links": ([_vp, _vp, _vp], _i),
    "stag_multishift_solve": ([_vp, _d, _i, _vp, _i, _i, _vp, _vp, _d, _i, C.POINTER(stag_solve_info)], _i),
    "stag_fermion_force": ([_vp, _d, C.POINTER(stag_rational), _i, _i, _vp, _vp, _d, _i,
                            C.POINTER(stag_solve_info)], _i),
    "stag_gauge_force": ([_vp, _d, _vp], _i),
    "stag_plaquette": ([_vp, C.POINTER(_d)], _i),
    "stag_md_trajectory": ([_vp, C.POINTER(stag_hmc), C.POINTER(stag_traj)], _i),
    "stag_multishift_solve_batch": ([C.POINTER(_vp), _i, _d, _i, _vp, _i, C.POINTER(_vp), C.POINTER(_vp), _d, _i,
                                     C.POINTER(stag_solve_info)], _i),
    "stag_selftest_barrier_timeout": ([_vp, C.c_longlong], _i),
    "stag_profile_batch_phases": ([_vp, _i, C.POINTER(_d)], _i),
    "stag_batch_shape": ([_vp, _i, C.POINTER(_i), C.POINTER(_i)], _i),
    "stag_md_trajectory_batch": ([C.POINTER(_vp), _i, C.POINTER(stag_hmc), C.POINTER(stag_traj)], _i),
    "stag_momenta": ([_vp], _vp),
    "stag_profile_begin": ([_vp, _i], _i),
    "stag_profile_read": ([_vp, _i, C.POINTER(stag_kernel_profile)], _i),
    "stag_launch_count": ([_vp], C.c_longlong),
    "stag_profile_phases": ([_vp, C.POINTER(_d)], _i),
    "stag_tuned_threads_per_site": ([_vp, _i, _i, C.POINTER(_d)], _i),
    "stag_surrogate_load": ([_vp, _vp], _i),
    "stag_surrogate_store": ([_vp, _vp], _i),
    "stag_surrogate_force": ([_vp, _vp], _i),
    "stag_surrogate_add_force_sample": ([_vp, _vp], _i),
    "stag_surrogate_add_sample": ([_vp, C.POINTER(stag_hmc), C.c_ulonglong], _i),
    "stag_surrogate_samples": ([_vp], C.c_longlong),
    "stag_surrogate_reserve": ([_vp, C.c_longlong], _i),
    "stag_surrogate_loss_grad": ([_vp, C.POINTER(_d), _vp], _i),
    "stag_surrogate_train": ([_vp, _i, _d, C.POINTER(_d), C.POINTER(_d)], _i),
    "stag_draw_momenta": ([_vp, C.c_ulonglong, C.c_ulonglong, _vp], _i),
    "stag_draw_sources": ([_vp, C.c_ulonglong, C.c_ulonglong, _i, _i, _vp], _i),
}

_lib = None
_keep = []   # ctypes arrays referenced by live structs


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libstag is not built ({LIB_PATH} missing); run "
                              "python -m paper_1010_5433_gb300.build")
        L = C.CDLL(LIB_PATH)
        sig = SIGNATURES
        for name, (args, res) in sig.items():
            if not hasattr(L, name):
                continue           # reported by the export test; calling it raises
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(t)}")


def _check(status, where, ctx=None):
    if status != 0:
        detail = ""
        if ctx is not None and status == 3:
            detail = lib().stag_last_cuda_error(ctx).decode()
        raise StagError(status, where, detail)
    return status


def _darr(vals):
    a = (C.c_double * max(1, len(vals)))(*vals)
    _keep.append(a)
    return a


def make_rational(a0, alpha, beta):
    r = stag_rational()
    r.n = len(alpha)
    r.a0 = float(a0)
    r.alpha = C.cast(_darr([float(v) for v in alpha]), C.POINTER(C.c_double))
    r.beta = C.cast(_darr([float(v) for v in beta]), C.POINTER(C.c_double))
    return r


# ---------------------------------------------------------------- C-named calls
def stag_create(dims, t_antiperiodic=True, cuda_stream=None):
    lat = stag_lattice()
    for k in range(4):
        lat.dims[k] = int(dims[k])
    lat.t_antiperiodic = 1 if t_antiperiodic else 0
    lat.cuda_stream = _ptr(cuda_stream) if cuda_stream is not None else None
    h = C.c_void_p()
    _check(lib().stag_create(C.byref(lat), C.byref(h)), "stag_create")
    return h


def stag_destroy(ctx):
    lib().stag_destroy(ctx)


def stag_set_stream(ctx, stream):
    _check(lib().stag_set_stream(ctx, _ptr(stream)), "stag_set_stream", ctx)


def stag_device_bytes(ctx):
    return lib().stag_device_bytes(ctx)


def stag_load_gauge(ctx, host_u):
    """host_u: C-contiguous float64 host array (numpy or CPU tensor), 4*V*18 values."""
    _check(lib().stag_load_gauge(ctx, _ptr(host_u)), "stag_load_gauge", ctx)


def stag_load_gauge_device(ctx, dev_u):
    _check(lib().stag_load_gauge_device(ctx, _ptr(dev_u)), "stag_load_gauge_device", ctx)


def stag_store_gauge(ctx, host_u):
    _check(lib().stag_store_gauge(ctx, _ptr(host_u)), "stag_store_gauge", ctx)


def stag_dslash(ctx, out_parity, prec, nrhs, inp, out):
    _check(lib().stag_dslash(ctx, int(out_parity), int(prec), int(nrhs), _ptr(inp), _ptr(out)), "stag_dslash", ctx)


def stag_apply_a(ctx, mass, shift, prec, nrhs, inp, out):
    _check(lib().stag_apply_a(ctx, float(mass), float(shift), int(prec), int(nrhs), _ptr(inp), _ptr(out)),
           "stag_apply_a", ctx)


def stag_apply_a_noalloc(ctx, mass, shift, prec, nrhs, inp, out):
    """stag_apply_a without any device allocation (fixed library scratch)."""
    st = lib().stag_apply_a_noalloc(ctx, float(mass), float(shift), int(prec), int(nrhs), _ptr(inp), _ptr(out))
    if st != 0:
        raise StagError(st, "stag_apply_a_noalloc", lib().stag_last_cuda_error(ctx).decode())


def stag_set_action(ctx, action, u0=1.0):
    """STAG_ACTION_UNIMPROVED (the paper's operator) or STAG_ACTION_ASQTAD with tadpole factor u0."""
    _check(lib().stag_set_action(ctx, int(action), float(u0)), "stag_set_action", ctx)


def stag_asqtad_links(ctx, host_fat, host_naik):
    """Fat and Naik links into float64 host arrays of 4*V*18 values each (host gauge layout)."""
    _check(lib().stag_asqtad_links(ctx, _ptr(host_fat), _ptr(host_naik)), "stag_asqtad_links", ctx)


def stag_multishift_solve(ctx, mass, shifts, prec, nrhs, b, x, tol, max_iter, info=True, check=True):
    sh = _darr([float(s) for s in shifts])
    inf = stag_solve_info() if info else None
    st = lib().stag_multishift_solve(ctx, float(mass), len(shifts), C.cast(sh, C.c_void_p), int(prec), int(nrhs),
                                     _ptr(b), _ptr(x), float(tol), int(max_iter),
                                     C.byref(inf) if inf is not None else None)
    if check:
        _check(st, "stag_multishift_solve", ctx)
    return (st, inf) if not check else inf


def stag_multishift_solve_batch(ctxs, mass, shifts, prec, bs, xs, tol, max_iter, check=True):
    """Solve (A + shift_i) x = b on every lattice (context) of ctxs at once; bs, xs device fp64 arrays."""
    n = len(ctxs)
    sh = _darr([float(s) for s in shifts])
    carr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    barr = (C.c_void_p * n)(*[_ptr(b) for b in bs])
    xarr = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    infos = (stag_solve_info * n)()
    st = lib().stag_multishift_solve_batch(carr, n, float(mass), len(shifts), C.cast(sh, C.c_void_p), int(prec),
                                           barr, xarr, float(tol), int(max_iter), infos)
    if check:
        _check(st, "stag_multishift_solve_batch", ctxs[0])
        return list(infos)
    return st, list(infos)


def stag_fermion_force(ctx, mass, rational, prec, n_pf, phi, force, tol, max_iter, info=True):
    inf = stag_solve_info() if info else None
    _check(lib().stag_fermion_force(ctx, float(mass), C.byref(rational), int(prec), int(n_pf), _ptr(phi),
                                    _ptr(force), float(tol), int(max_iter),
                                    C.byref(inf) if inf is not None else None), "stag_fermion_force", ctx)
    return inf


def stag_gauge_force(ctx, beta, force):
    _check(lib().stag_gauge_force(ctx, float(beta), _ptr(force)), "stag_gauge_force", ctx)


def stag_plaquette(ctx):
    v = C.c_double()
    _check(lib().stag_plaquette(ctx, C.byref(v)), "stag_plaquette", ctx)
    return v.value


def stag_md_trajectory(ctx, hmc):
    out = stag_traj()
    st = lib().stag_md_trajectory(ctx, C.byref(hmc), C.byref(out))
    _check(st, "stag_md_trajectory", ctx)
    return out


def stag_md_trajectory_batch(ctxs, hmcs):
    """One trajectory of each chain (context) in ctxs with parameters hmcs, advanced together."""
    n = len(ctxs)
    carr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    harr = (stag_hmc * n)(*hmcs)
    outs = (stag_traj * n)()
    _check(lib().stag_md_trajectory_batch(carr, n, harr, outs), "stag_md_trajectory_batch", ctxs[0])
    return list(outs)


def stag_momenta(ctx):
    return lib().stag_momenta(ctx)


def stag_draw_momenta(ctx, seed, counter, mom):
    _check(lib().stag_draw_momenta(ctx, int(seed), int(counter), _ptr(mom)), "stag_draw_momenta", ctx)


def stag_draw_sources(ctx, seed, counter, stream, n, xi):
    _check(lib().stag_draw_sources(ctx, int(seed), int(counter), int(stream), int(n), _ptr(xi)),
           "stag_draw_sources", ctx)


STAG_PK_DSLASH_OE, STAG_PK_DSLASH_EO_A, STAG_PK_UPDATE, STAG_PK_PERSISTENT, STAG_PK_BATCH, STAG_PK_PERSISTENT_FF = \
    0, 1, 2, 3, 4, 5


def stag_profile_begin(ctx, sample_every):
    _check(lib().stag_profile_begin(ctx, int(sample_every)), "stag_profile_begin", ctx)


def stag_profile_read(ctx, kind):
    out = stag_kernel_profile()
    _check(lib().stag_profile_read(ctx, int(kind), C.byref(out)), "stag_profile_read", ctx)
    return out


def stag_selftest_barrier_timeout(ctx, spin_limit):
    """Status of the barrier self-test (STAG_ERR_TIMEOUT = 5 when the bounded wait gave up)."""
    return lib().stag_selftest_barrier_timeout(ctx, int(spin_limit))


def stag_profile_batch_phases(ctx, prec):
    us = (C.c_double * 8)()
    _check(lib().stag_profile_batch_phases(ctx, int(prec), us), "stag_profile_batch_phases", ctx)
    return list(us)


def stag_batch_shape(ctx, prec):
    """(index, threads per block, blocks per SM) of the tuned batched-solver launch shape; index -1 while tuning."""
    a, b = C.c_int(0), C.c_int(0)
    k = lib().stag_batch_shape(ctx, int(prec), C.byref(a), C.byref(b))
    return k, a.value, b.value


def stag_launch_count(ctx):
    return lib().stag_launch_count(ctx)


def stag_tuned_threads_per_site(ctx, prec, nrhs):
    us = C.c_double()
    t = lib().stag_tuned_threads_per_site(ctx, int(prec), int(nrhs), C.byref(us))
    return t, us.value


def stag_profile_phases(ctx):
    arr = (C.c_double * 15)()
    _check(lib().stag_profile_phases(ctx, arr), "stag_profile_phases", ctx)
    return list(arr)


STAG_SUR_PARAMS = 2648


def stag_surrogate_load(ctx, params):
    """params: host float32 array (numpy) of STAG_SUR_PARAMS values."""
    _check(lib().stag_surrogate_load(ctx, _ptr(params)), "stag_surrogate_load", ctx)


def stag_surrogate_store(ctx, params):
    _check(lib().stag_surrogate_store(ctx, _ptr(params)), "stag_surrogate_store", ctx)


def stag_surrogate_force(ctx, force):
    _check(lib().stag_surrogate_force(ctx, _ptr(force)), "stag_surrogate_force", ctx)


def stag_surrogate_add_force_sample(ctx, force):
    _check(lib().stag_surrogate_add_force_sample(ctx, _ptr(force)), "stag_surrogate_add_force_sample", ctx)


def stag_surrogate_add_sample(ctx, hmc, counter):
    _check(lib().stag_surrogate_add_sample(ctx, C.byref(hmc), int(counter)), "stag_surrogate_add_sample", ctx)


def stag_surrogate_samples(ctx):
    return lib().stag_surrogate_samples(ctx)


def stag_surrogate_reserve(ctx, n_samples):
    _check(lib().stag_surrogate_reserve(ctx, int(n_samples)), "stag_surrogate_reserve", ctx)


def stag_surrogate_loss_grad(ctx, grad=None):
    loss = C.c_double()
    _check(lib().stag_surrogate_loss_grad(ctx, C.byref(loss), _ptr(grad)), "stag_surrogate_loss_grad", ctx)
    return loss.value


def stag_surrogate_train(ctx, steps, lr):
    a, b = C.c_double(), C.c_double()
    _check(lib().stag_surrogate_train(ctx, int(steps), float(lr), C.byref(a), C.byref(b)), "stag_surrogate_train", ctx)
    return a.value, b.value
