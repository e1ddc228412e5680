"""Python binding of libdns.so, the GB300 ensemble channel-DNS step library.

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  PyTorch provides the device workspace and the CUDA stream.

Functions named ``dns_*`` mirror the C ABI in ``include/dns.h`` one to one;
``Ensemble`` is a convenience wrapper around them.  Importing this package
raises ImportError if ``libdns.so`` has not been built (run
``python -c "import __graft_entry__ as g; g.build()"``); there is no fallback.
"""
import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DNS_CHECKED=1 loads the bounds-checked debug build instead (built by
# paper_2306_12739_gb300/build.py with checked=True)
LIB_PATH = os.path.join(_HERE, "libdns_check.so" if os.environ.get("DNS_CHECKED") == "1" else "libdns.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libdns.so is not built at %s; build it with paper_2306_12739_gb300.build" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)

DNS_OK = 0
DNS_ERR_INVALID = -1
DNS_ERR_CUDA = -2
DNS_ERR_NOMEM = -3
DNS_ERR_TIMEOUT = -4
DNS_ERR_NONFINITE = -5
DNS_ERR_UNSUPPORTED = -6
DNS_COUETTE, DNS_POISEUILLE = 0, 1
DNS_PREC_FP64, DNS_PREC_MIXED = 0, 1

EXPORTED = ["dns_create", "dns_workspace_size", "dns_bind_workspace", "dns_state_shape",
            "dns_set_state", "dns_get_state", "dns_step", "dns_stats", "dns_destroy",
            "dns_last_error", "dns_last_launch_count", "dns_export_grid", "dns_export_operators",
            "dns_step_timed", "dns_stats_noalloc", "dns_selftest_timeout", "dns_kernel_choice",
            "dns_convert_selftest", "dns_set_base_flow", "dns_set_direction", "dns_orthonormalize",
            "dns_optimal_sweep", "dns_set_stochastic_forcing", "dns_export_forcing", "dns_advance",
            "dns_checked_build", "dns_selftest_bounds"]
KERNEL_CLASSES = ["mean_deriv", "yderiv", "plane", "forcing", "helm", "mean", "spec", "d2v"]


class dns_group_desc(ctypes.Structure):
    _fields_ = [("flow", ctypes.c_int), ("mx", ctypes.c_int), ("my", ctypes.c_int), ("mz", ctypes.c_int),
                ("lx", ctypes.c_double), ("lz", ctypes.c_double), ("re", ctypes.c_double),
                ("dt", ctypes.c_double), ("u_wall", ctypes.c_double), ("bulk_flux", ctypes.c_double),
                ("members", ctypes.c_int), ("shared_mean", ctypes.c_int), ("nonlinear_form", ctypes.c_int),
                ("member_block", ctypes.c_int), ("linear", ctypes.c_int), ("kx_index", ctypes.c_int)]


class dns_config(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int), ("groups", ctypes.POINTER(dns_group_desc)),
                ("precision", ctypes.c_int), ("use_graph", ctypes.c_int), ("persistent", ctypes.c_int),
                ("barrier_timeout_ns", ctypes.c_ulonglong), ("autotune_cache", ctypes.c_char_p),
                ("ygemm", ctypes.c_int), ("plane", ctypes.c_int), ("helm", ctypes.c_int)]


class dns_stats_t(ctypes.Structure):
    _fields_ = [("e_total", ctypes.c_double), ("e_pert", ctypes.c_double), ("tau_bottom", ctypes.c_double),
                ("tau_top", ctypes.c_double), ("bulk_flux", ctypes.c_double), ("gamma", ctypes.c_double),
                ("max_div", ctypes.c_double), ("nonfinite", ctypes.c_int), ("reserved", ctypes.c_int),
                ("cfl", ctypes.c_double)]


class dns_state_in(ctypes.Structure):
    _fields_ = [("v_hat", ctypes.c_void_p), ("eta_hat", ctypes.c_void_p), ("U00", ctypes.c_void_p),
                ("W00", ctypes.c_void_p)]


class dns_state_out(ctypes.Structure):
    _fields_ = [("v_hat", ctypes.c_void_p), ("eta_hat", ctypes.c_void_p), ("U00", ctypes.c_void_p),
                ("W00", ctypes.c_void_p)]


_H = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p

_lib.dns_create.argtypes = [ctypes.POINTER(dns_config), _vp, ctypes.POINTER(_H)]
_lib.dns_workspace_size.argtypes = [_H, ctypes.POINTER(ctypes.c_size_t)]
_lib.dns_bind_workspace.argtypes = [_H, _vp, ctypes.c_size_t]
_lib.dns_state_shape.argtypes = [_H, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4
_lib.dns_set_state.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int]
_lib.dns_get_state.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int]
_lib.dns_step.argtypes = [_H, ctypes.c_int]
_lib.dns_advance.argtypes = [_H, ctypes.c_int, ctypes.POINTER(dns_state_in), ctypes.POINTER(dns_state_out),
                             ctypes.c_int]
_lib.dns_stats.argtypes = [_H, ctypes.c_int, ctypes.POINTER(dns_stats_t), ctypes.POINTER(dns_stats_t), _dp]
_lib.dns_destroy.argtypes = [_H]
_lib.dns_last_error.argtypes = [_H]
_lib.dns_last_error.restype = ctypes.c_char_p
_lib.dns_last_launch_count.argtypes = [_H]
_lib.dns_step_timed.argtypes = [_H, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int)]
_lib.dns_stats_noalloc.argtypes = [_H, ctypes.c_int, _vp]
_lib.dns_selftest_timeout.argtypes = [_H]
_lib.dns_selftest_bounds.argtypes = [_H]
_lib.dns_checked_build.argtypes = []
_lib.dns_convert_selftest.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_longlong]
_lib.dns_kernel_choice.argtypes = [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]
_lib.dns_export_grid.argtypes = [_H, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
_lib.dns_export_operators.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
_lib.dns_set_base_flow.argtypes = [_H, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int]
_lib.dns_set_direction.argtypes = [_H, ctypes.c_int, ctypes.c_int]
_lib.dns_orthonormalize.argtypes = [_H, ctypes.c_int, _vp]
_lib.dns_optimal_sweep.argtypes = [_H, ctypes.c_int, _vp]
_lib.dns_set_stochastic_forcing.argtypes = [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_ulonglong]
_lib.dns_export_forcing.argtypes = [_H, ctypes.c_int, ctypes.c_int, _vp, _vp]


class DnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dns error %d: %s" % (code, msg))
        self.code = code


def _ck(h, rc):
    if rc != DNS_OK:
        msg = _lib.dns_last_error(h)
        raise DnsError(rc, msg.decode() if msg else "")
    return rc


# ------------------------------------------------------------ C-ABI mirror

def dns_create(cfg, stream=0):
    h = _H()
    rc = _lib.dns_create(ctypes.byref(cfg), _vp(stream), ctypes.byref(h))
    if rc != DNS_OK:
        msg = _lib.dns_last_error(h).decode() if h.value else ""
        if h.value:
            _lib.dns_destroy(h)
        raise DnsError(rc, msg)
    return h


def dns_workspace_size(h):
    n = ctypes.c_size_t()
    _ck(h, _lib.dns_workspace_size(h, ctypes.byref(n)))
    return n.value


def dns_bind_workspace(h, ptr, nbytes):
    return _ck(h, _lib.dns_bind_workspace(h, _vp(ptr), nbytes))


def dns_state_shape(h, group):
    a = [ctypes.c_int() for _ in range(4)]
    _ck(h, _lib.dns_state_shape(h, group, *[ctypes.byref(x) for x in a]))
    return tuple(x.value for x in a)


def dns_set_state(h, group, member0, count, v, eta, U, W, ptr_kind):
    return _ck(h, _lib.dns_set_state(h, group, member0, count, _vp(v), _vp(eta), _vp(U), _vp(W), ptr_kind))


def dns_get_state(h, group, member0, count, v, eta, U, W, ptr_kind):
    return _ck(h, _lib.dns_get_state(h, group, member0, count, _vp(v), _vp(eta), _vp(U), _vp(W), ptr_kind))


def dns_step(h, nsteps):
    return _ck(h, _lib.dns_step(h, nsteps))


def dns_advance(h, nsteps, ins, outs, ptr_kind):
    """ins, outs: one (v, eta, U, W) tuple of raw addresses (or None) per group,
    or None for the whole argument (no upload / no download)."""
    pin = (dns_state_in * len(ins))(*[dns_state_in(*a) for a in ins]) if ins is not None else None
    pout = (dns_state_out * len(outs))(*[dns_state_out(*a) for a in outs]) if outs is not None else None
    return _ck(h, _lib.dns_advance(h, nsteps, pin, pout, ptr_kind))


def dns_step_timed(h, nsteps):
    """Returns {kernel class: (total ms, launches)} over nsteps eager steps."""
    ms = (ctypes.c_double * len(KERNEL_CLASSES))()
    n = (ctypes.c_int * len(KERNEL_CLASSES))()
    _ck(h, _lib.dns_step_timed(h, nsteps, ms, n))
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES)}


def dns_stats(h, group, members, profiles_ptr=None):
    per = (dns_stats_t * members)()
    mean = dns_stats_t()
    rc = _lib.dns_stats(h, group, per, ctypes.byref(mean),
                        ctypes.cast(profiles_ptr, _dp) if profiles_ptr else None)
    if rc not in (DNS_OK, DNS_ERR_NONFINITE):
        _ck(h, rc)
    return rc, per, mean


def dns_stats_noalloc(h, group, out_dev_ptr):
    """Allocation-free statistics into a caller-owned DEVICE buffer
    [members][8] (see include/dns.h); asynchronous on the handle's stream."""
    return _ck(h, _lib.dns_stats_noalloc(h, group, _vp(out_dev_ptr)))


def dns_checked_build():
    """1 when the loaded library is the bounds-checked debug build."""
    return _lib.dns_checked_build()


def dns_selftest_bounds(h):
    """Records one failing bounds check (no memory touched) and synchronises;
    returns the status code (DNS_ERR_CUDA in the checked build, DNS_OK
    otherwise) without raising."""
    return _lib.dns_selftest_bounds(h)


def dns_selftest_timeout(h):
    """Runs a bounded device wait that must give up; returns the status code
    (DNS_ERR_TIMEOUT expected) without raising."""
    return _lib.dns_selftest_timeout(h)


def convert_selftest(d_in, f_in):
    """Host run of the library's integer binary64 -> binary32 (round to nearest
    even) and binary32 -> binary64 conversions; returns (f_out, d_out)."""
    import numpy as np
    d_in = np.ascontiguousarray(d_in, dtype=np.float64)
    f_in = np.ascontiguousarray(f_in, dtype=np.float32)
    assert d_in.shape == f_in.shape
    f_out = np.empty_like(f_in)
    d_out = np.empty_like(d_in)
    rc = _lib.dns_convert_selftest(d_in.ctypes.data, f_out.ctypes.data, f_in.ctypes.data, d_out.ctypes.data,
                                   d_in.size)
    if rc != DNS_OK:
        raise DnsError(rc, "dns_convert_selftest")
    return f_out, d_out


def dns_kernel_choice(h, group, which="ygemm"):
    """'ygemm' -> 'simt' | 'tc' | 'simt_eo'; 'plane' -> 'cta' | 'cluster' | 'lines' | 'linear';
    'helm' -> 'simt' | 'tc' | 'persist' | 'fused' | 'fused_d2v' | 'fused_eo' | 'fused_eo_ff' | 'simt_eo'."""
    c, p, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _ck(h, _lib.dns_kernel_choice(h, group, ctypes.byref(c), ctypes.byref(p), ctypes.byref(m)))
    # the names of the request tables (one source for both directions); plane 4,
    # the linearised groups' own kernel, is never requested
    if which == "plane":
        return {**_names(_PLANE), 4: "linear"}.get(p.value, p.value)
    if which == "helm":
        return _names(_HELM).get(m.value, m.value)
    return _names(_YGEMM).get(c.value, c.value)


def _names(table):
    """number -> name of a request table, without the autotune aliases."""
    return {v: k for k, v in table.items() if v != 0}


def dns_set_base_flow(h, group, U, V, W, ptr_kind):
    return _ck(h, _lib.dns_set_base_flow(h, group, _vp(U), _vp(V), _vp(W), ptr_kind))


def dns_set_direction(h, group, adjoint):
    return _ck(h, _lib.dns_set_direction(h, group, 1 if adjoint else 0))


def dns_orthonormalize(h, group, norms_ptr=None):
    return _ck(h, _lib.dns_orthonormalize(h, group, _vp(norms_ptr) if norms_ptr else None))


def dns_optimal_sweep(h, nsteps, gains_ptr=None):
    return _ck(h, _lib.dns_optimal_sweep(h, nsteps, _vp(gains_ptr) if gains_ptr else None))


def dns_set_stochastic_forcing(h, group, kx_index, n_eig, rate, seed):
    return _ck(h, _lib.dns_set_stochastic_forcing(h, group, kx_index, n_eig, float(rate), int(seed)))


def dns_export_forcing(h, group, m_index, n_eig, ny):
    f = np.zeros((2, n_eig, ny))
    lam = np.zeros((2, n_eig))
    _ck(h, _lib.dns_export_forcing(h, group, m_index, f.ctypes.data, lam.ctypes.data))
    return f, lam


def dns_destroy(h):
    return _lib.dns_destroy(h)


def dns_last_error(h):
    return _lib.dns_last_error(h).decode()


def dns_last_launch_count(h):
    return _lib.dns_last_launch_count(h)


def dns_export_grid(h, group, my):
    y = np.zeros(my); D1 = np.zeros((my, my)); D2 = np.zeros((my, my))
    D4 = np.zeros((my - 2, my - 2)); w = np.zeros(my)
    p = lambda a: a.ctypes.data_as(_dp)
    _ck(h, _lib.dns_export_grid(h, group, p(y), p(D1), p(D2), p(D4), p(w)))
    return y, D1, D2, D4, w


def dns_export_operators(h, group, h_index, pair, ny):
    out = [np.zeros((ny, ny)) for _ in range(4)]
    _ck(h, _lib.dns_export_operators(h, group, h_index, pair, *[a.ctypes.data_as(_dp) for a in out]))
    return out


# ---------------------------------------------------------------- wrapper

_FLOWS = {"couette": DNS_COUETTE, "poiseuille": DNS_POISEUILLE}
_PRECS = {"fp64": DNS_PREC_FP64, "mixed": DNS_PREC_MIXED}


_YGEMM = {"default": 0, "auto": 0, "simt": 1, "tc": 2, "simt_eo": 3}


_PLANE = {"default": 0, "auto": 0, "cta": 1, "cluster": 2, "lines": 3}


_HELM = {"default": 0, "auto": 0, "simt": 1, "tc": 2, "persist": 3, "fused": 4, "fused_d2v": 5, "fused_eo": 6, "fused_eo_ff": 7, "simt_eo": 8}


def _pick(table, name, what):
    try:
        return table[name]
    except KeyError:
        raise ValueError("unknown %s %r (choices: %s)" % (what, name, ", ".join(sorted(table)))) from None


def make_config(groups, precision="fp64", use_graph=False, ygemm="default", autotune_cache=None, plane="default",
                helm="default"):
    """groups: list of dicts with flow, mx, my, mz, lx, lz, re, dt, members,
    optional u_wall (1.0), bulk_flux (4/3), shared_mean (False; True: the
    members share their kx = 0 flow, S3T-type ensemble), form ("advective"
    or "rotational" nonlinear term), member_block (0: automatic size of the
    concurrently run member blocks), linear (True: a linearised disturbance
    ensemble of one streamwise wavenumber) and kx_index (its n >= 1).
    autotune_cache: file of kernel-variant decisions read and appended at bind
    time (None: the DNS_AUTOTUNE_CACHE environment variable, if set).
    ygemm, plane, helm: kernel-variant requests of the mixed path ("default":
    autotuned at bind time; dns_config in include/dns.h describes each):
    ygemm simt | tc | simt_eo; plane cta | cluster | lines; helm simt | tc |
    persist | fused | fused_d2v | fused_eo | fused_eo_ff | simt_eo."""
    arr = (dns_group_desc * len(groups))()
    for i, g in enumerate(groups):
        arr[i] = dns_group_desc(_pick(_FLOWS, g["flow"], "flow"), g["mx"], g["my"], g["mz"], g["lx"], g["lz"], g["re"],
                                g["dt"], g.get("u_wall", 1.0), g.get("bulk_flux", 4.0 / 3.0), g["members"],
                                1 if g.get("shared_mean", False) else 0,
                                _pick({"advective": 0, "rotational": 1}, g.get("form", "advective"), "form"),
                                int(g.get("member_block", 0)), 1 if g.get("linear", False) else 0,
                                int(g.get("kx_index", 0)))
    if autotune_cache is None:      # the environment may name a cache shared by every handle
        autotune_cache = os.environ.get("DNS_AUTOTUNE_CACHE") or None
    cache = autotune_cache.encode() if autotune_cache else None
    cfg = dns_config(len(groups), arr, _pick(_PRECS, precision, "precision"), 1 if use_graph else 0, 0, 0, cache,
                     _pick(_YGEMM, ygemm, "ygemm variant"), _pick(_PLANE, plane, "plane variant"),
                     _pick(_HELM, helm, "helm variant"))
    cfg._keep = (arr, cache)
    return cfg


# ------------------------------------------------------------- checkpoints

_STATE_KEYS = ("v", "eta", "U", "W")


def save_states(path, groups, states):
    """Checkpoint file (.npz): the group descriptions (as JSON) and every
    group's state (v, eta, U, W in the host layout; U, W None for a linear
    group), written exactly (no conversion)."""
    arrs = {"groups": np.array(json.dumps(groups))}
    for i, st in enumerate(states):
        for k, a in zip(_STATE_KEYS, st):
            if a is not None:
                arrs["g%d_%s" % (i, k)] = np.asarray(a)
    np.savez(path, **arrs)


def load_states(path):
    """(groups, states) of a checkpoint written by save_states."""
    with np.load(path, allow_pickle=False) as z:
        groups = json.loads(str(z["groups"]))
        states = [tuple(z["g%d_%s" % (i, k)] if "g%d_%s" % (i, k) in z.files else None for k in _STATE_KEYS)
                  for i in range(len(groups))]
    return groups, states


def same_groups(a, b):
    """True when two lists of group descriptions describe the same groups (as a
    checkpoint stores them)."""
    return json.loads(json.dumps(a)) == json.loads(json.dumps(b))


class Ensemble:
    """Owns a handle, its torch workspace and the stream it runs on."""

    def __init__(self, groups, precision="fp64", use_graph=False, device="cuda:0", stream=None, ygemm="default",
                 autotune_cache=None, plane="default", helm="default"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.groups = [dict(g) for g in groups]
        # a stream of its own: graph capture is not allowed on the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.cfg = make_config(groups, precision, use_graph, ygemm, autotune_cache, plane, helm)
        self.h = dns_create(self.cfg, self.stream.cuda_stream)
        nbytes = dns_workspace_size(self.h)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self.ws_ptr = (base + 255) & ~255
        dns_bind_workspace(self.h, self.ws_ptr, nbytes)
        self.shapes = [dns_state_shape(self.h, i) for i in range(len(groups))]

    def close(self):
        if self.h is not None:
            dns_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, group, v, eta, U=None, W=None, member0=0):
        """v, eta complex128 [count][Ny][NKZ][NKX]; U, W float64 [count][My]
        (None for a linear group, whose NKX is 1 and which has no mean profiles).
        numpy arrays (host) or torch CUDA tensors (device, complex128/float64)."""
        torch = self.torch
        if U is None or W is None:
            nkx, nkz, ny, _ = self.shapes[group]
            arrs = [np.ascontiguousarray(np.reshape(a, (-1, ny, nkz, nkx)), dtype=np.complex128) for a in (v, eta)]
            dns_set_state(self.h, group, member0, arrs[0].shape[0], arrs[0].ctypes.data, arrs[1].ctypes.data,
                          None, None, 0)
            return
        if isinstance(v, torch.Tensor):
            ts = [t.contiguous() for t in (v, eta, U, W)]
            count = ts[0].shape[0]
            dns_set_state(self.h, group, member0, count, *[t.data_ptr() for t in ts], 1)
            self._keep = ts
        else:
            arrs = [np.ascontiguousarray(v, dtype=np.complex128), np.ascontiguousarray(eta, dtype=np.complex128),
                    np.ascontiguousarray(U, dtype=np.float64), np.ascontiguousarray(W, dtype=np.float64)]
            count = arrs[0].shape[0]
            dns_set_state(self.h, group, member0, count, *[a.ctypes.data for a in arrs], 0)

    def get_state(self, group, member0=0, count=None):
        nkx, nkz, ny, my = self.shapes[group]
        if count is None:
            count = self.groups[group]["members"] - member0
        v = np.zeros((count, ny, nkz, nkx), dtype=np.complex128)
        e = np.zeros_like(v)
        U = np.zeros((count, my)); W = np.zeros((count, my))
        dns_get_state(self.h, group, member0, count, v.ctypes.data, e.ctypes.data, U.ctypes.data,
                      W.ctypes.data, 0)
        return v, e, U, W

    def step(self, nsteps=1):
        dns_step(self.h, nsteps)

    def checkpoint(self, path):
        """Write every group's current state to a checkpoint file (save_states)."""
        save_states(path, self.groups, [self.get_state(i) for i in range(len(self.groups))])

    def restore(self, path):
        """Set every group's state from a checkpoint of the same groups."""
        groups, states = load_states(path)
        if not same_groups(groups, self.groups):
            raise ValueError("the checkpoint holds other groups")
        for i, st in enumerate(states):
            if self.groups[i].get("linear"):
                self.set_state(i, st[0], st[1])
            else:
                self.set_state(i, *st)

    def advance(self, nsteps, states):
        """Replace every group's state by states[group] = (v, eta, U, W) (host
        numpy arrays, U and W None for a linear group), advance nsteps steps and
        return the new states, in one dns_advance call."""
        ins, outs, res = [], [], []
        for gi, st in enumerate(states):
            nkx, nkz, ny, my = self.shapes[gi]
            E = self.groups[gi]["members"]
            v = np.ascontiguousarray(np.reshape(st[0], (E, ny, nkz, nkx)), dtype=np.complex128)
            e = np.ascontiguousarray(np.reshape(st[1], (E, ny, nkz, nkx)), dtype=np.complex128)
            U = None if st[2] is None else np.ascontiguousarray(st[2], dtype=np.float64)
            W = None if st[3] is None else np.ascontiguousarray(st[3], dtype=np.float64)
            o = (np.zeros_like(v), np.zeros_like(e), np.zeros((E, my)), np.zeros((E, my)))
            ins.append((v, e, U, W))
            res.append(o)
            outs.append(o)
        addr = lambda a: a.ctypes.data if a is not None else None
        dns_advance(self.h, nsteps, [tuple(addr(a) for a in t) for t in ins],
                    [tuple(addr(a) for a in t) for t in outs], 0)
        return res

    def set_stochastic_forcing(self, group, kx_index, n_eig, rate, seed):
        dns_set_stochastic_forcing(self.h, group, kx_index, n_eig, rate, seed)

    # ---- linearised disturbance groups
    def set_base_flow(self, group, U, V, W):
        """U, V, W float64 [My][Mz] on the Chebyshev nodes x uniform z (host)."""
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (U, V, W)]
        dns_set_base_flow(self.h, group, a[0].ctypes.data, a[1].ctypes.data, a[2].ctypes.data, 0)

    def set_direction(self, adjoint, group=-1):
        dns_set_direction(self.h, group, adjoint)

    def orthonormalize(self, group):
        """Energy-norm modified Gram-Schmidt of the group's members; returns the
        norms before normalisation."""
        r = np.zeros(self.groups[group]["members"])
        dns_orthonormalize(self.h, group, r.ctypes.data)
        return r

    def optimal_sweep(self, nsteps):
        """One forward-adjoint iteration of every (linear) group; returns the
        gains per group."""
        sizes = [g["members"] for g in self.groups]
        out = np.zeros(sum(sizes))
        dns_optimal_sweep(self.h, nsteps, out.ctypes.data)
        return np.split(out, np.cumsum(sizes)[:-1])

    def step_timed(self, nsteps=1):
        return dns_step_timed(self.h, nsteps)

    def launches(self):
        return dns_last_launch_count(self.h)

    def stats(self, group):
        E = self.groups[group]["members"]
        my = self.shapes[group][3]
        prof = np.zeros((E, 6, my))
        rc, per, mean = dns_stats(self.h, group, E, prof.ctypes.data)
        keys = [k for k, _ in dns_stats_t._fields_ if k != "reserved"]
        out = {k: np.array([getattr(per[i], k) for i in range(E)]) for k in keys}
        out.update({"U": prof[:, 0], "W": prof[:, 1], "uu": prof[:, 2], "vv": prof[:, 3],
                    "ww": prof[:, 4], "uv": prof[:, 5], "rc": rc})
        return out
