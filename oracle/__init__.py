"""FP64 CPU oracle for the tangent-point energy (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, FP64,
``-O2 -ffp-contract=off``, OpenMP over targets) with ctypes; the library is
compiled by :func:`build` and shares no code with the CUDA library.

Every function follows the definition it names (see ``oracle.c``):
Eq. (TP) and alpha = 6 in Sec. 2.2.2 for the energy, the chain rule of the
discrete sum (the structure of Eq. (dTP) / Eq. (dTP_reordered), Sec. 3.2)
for the gradient, and the inner-integral clustering of Sec. 3.2 for the
Barnes-Hut form.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` (and the MLP reference) into ``liboracle.so``."""
    srcs = [os.path.join(_HERE, f) for f in ("oracle.c", "oracle_mlp.c", "oracle_conf.c", "oracle_quad.c",
                                              "oracle_dt.c") if os.path.exists(os.path.join(_HERE, f))]
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "oracle.h")]):
        return _SO
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", _SO + ".tmp"] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_SO)
    i64, i32, dbl = C.c_int64, C.c_int, C.c_double
    lib.or_tri_data.argtypes = [_d, _i32, i64, _d, _d, _d]
    lib.or_energy.argtypes = [_d, _d, _d, _i32, i64, dbl, dbl, dbl, i32, i32]
    lib.or_energy.restype = dbl
    lib.or_admitted_pairs.argtypes = [_i32, i64, i32, i32]
    lib.or_admitted_pairs.restype = i64
    lib.or_energy_touching.argtypes = [_d, _d, _d, _i32, i64, _u8, dbl, dbl, dbl, i32, i32]
    lib.or_energy_touching.restype = dbl
    lib.or_tri_accum.argtypes = [_d, _d, _d, _i32, i64, C.c_void_p, i64, dbl, dbl, i32, _d, _d, _d, i32]
    lib.or_adjoint.argtypes = [_d, _i32, C.c_void_p, i64, _d, _d, _d, dbl, _d]
    lib.or_lbvh.argtypes = [_d, i64, i32, i32, _u32, _i32, _i32, _i32, _i32, _i32, _i32, _i32, C.POINTER(C.c_int64)]
    lib.or_lbvh.restype = i32
    lib.or_moments.argtypes = [_d, _i32, _d, _d, _d, i64, _i32, _i32, _i32, _d, _d]
    lib.or_bh_accum.argtypes = [_d, _d, _d, _i32, i64, _i32, _i32, _i32, _i32, _i32, _i32, i64, _d, _d, dbl, i32,
                                dbl, dbl, i32, _d, _d, _d, C.POINTER(C.c_int64), C.POINTER(C.c_int64), i32]
    lib.or_dt_accum.argtypes = [_d, _d, _d, _i32, i64, _i32, _i32, _i32, _i32, _i32, _i32, _d, _d, dbl, i32, dbl,
                                dbl, i32, _d, _d, _d, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64)]
    lib.or_dt_accum.restype = dbl
    lib.or_conf_energy.argtypes = [_d, _d, _d, i64, _d, _d, i64, dbl, dbl, dbl, i32]
    lib.or_conf_energy.restype = dbl
    lib.or_conf_accum.argtypes = [_d, _d, _d, i64, _d, _d, i64, dbl, dbl, _d, _d, _d, i32]
    lib.or_quad_points.argtypes = [_d, _i32, i64, i32, _d, _d, _d, _d, _d, _i32]
    lib.or_quad_adjoint.argtypes = [_d, _i32, i64, i32, _d, _d, _d, _d, _d, dbl, _d]
    if hasattr(lib, "or_mlp_forward"):
        _bind_mlp(lib)
    _lib = lib
    return lib


def _bind_mlp(lib):
    i64, i32, dbl = C.c_int64, C.c_int, C.c_double
    lib.or_mlp_nparam.restype = i64
    lib.or_mlp_forward.argtypes = [_d, i64, _d, _d]
    lib.or_mlp_backward.argtypes = [_d, i64, _d, _d, _d]
    lib.or_mlp_loss.argtypes = [i64, _d, _d, _d, C.c_void_p]
    lib.or_mlp_loss.restype = dbl
    lib.or_adamw_step.argtypes = [_d, _d, _d, _d, i64, dbl, dbl, dbl, dbl, dbl, i32]
    lib.or_far_features.argtypes = [_d, _d, _d, _d, _d]
    lib.or_far_channels.argtypes = [_d, _d, _d, _i64, i64, _i64, i64, _d, dbl, dbl, _d, _d]


def nthreads_default() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _prep(V, F):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    return V, F


def tri_data(V, F):
    """Centroids x [nt,3], unit normals nu [nt,3], areas w [nt] (FP64)."""
    lib = _load()
    V, F = _prep(V, F)
    nt = F.shape[0]
    x = np.zeros((nt, 3))
    nu = np.zeros((nt, 3))
    w = np.zeros(nt)
    lib.or_tri_data(V, F, nt, x, nu, w)
    return x, nu, w


def energy_soa(x, nu, w, F, q=6.0, p=12.0, c=1.0, adj=0, nthreads=None):
    """Phi from given per-triangle (x, nu, w); exclusion from the faces F."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    return lib.or_energy(x, nu, w, F, F.shape[0], q, p, c, adj, nthreads or nthreads_default())


def energy(V, F, q=6.0, p=12.0, c=1.0, adj=0, nthreads=None):
    """Phi = c * sum over admitted ordered pairs (Eq. TP, one centroid point per triangle)."""
    x, nu, w = tri_data(V, F)
    return energy_soa(x, nu, w, F, q, p, c, adj, nthreads)


def admitted_pairs(F, adj=0, nthreads=None):
    """Ordered pairs (T, S), T != S, that the sum of Eq. TP keeps (brute force over all nt^2 pairs)."""
    lib = _load()
    F = np.ascontiguousarray(F, dtype=np.int32)
    return int(lib.or_admitted_pairs(F, F.shape[0], adj, nthreads or nthreads_default()))


def energy_touching(V, F, tris, q=6.0, p=12.0, c=1.0, adj=0, nthreads=None):
    """The part of Phi from ordered pairs with at least one triangle in ``tris``."""
    lib = _load()
    V, F = _prep(V, F)
    x, nu, w = tri_data(V, F)
    in_set = np.zeros(F.shape[0], dtype=np.uint8)
    in_set[np.asarray(tris, dtype=np.int64)] = 1
    return lib.or_energy_touching(x, nu, w, F, F.shape[0], in_set, q, p, c, adj, nthreads or nthreads_default())


def tri_accum(V, F, tris=None, q=6.0, p=12.0, adj=0, nthreads=None, soa=None):
    """Per-triangle dPhi/dw_T, dPhi/dnu_T [.,3], dPhi/dx_T [.,3] (without c).

    ``tris`` selects triangles (all when None); ``soa`` = (x, nu, w) overrides
    the per-triangle data computed from V.
    """
    lib = _load()
    V, F = _prep(V, F)
    x, nu, w = soa if soa is not None else tri_data(V, F)
    x, nu, w = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, nu, w))
    if tris is None:
        m = F.shape[0]
        ptr = None
        lst = None
    else:
        lst = np.ascontiguousarray(tris, dtype=np.int64)
        m = lst.shape[0]
        ptr = lst.ctypes.data_as(C.c_void_p)
    gw = np.zeros(m)
    gnu = np.zeros((m, 3))
    gx = np.zeros((m, 3))
    lib.or_tri_accum(x, nu, w, F, F.shape[0], ptr, m, q, p, adj, gw, gnu, gx, nthreads or nthreads_default())
    return gw, gnu, gx


def adjoint(V, F, gw, gnu, gx, c=1.0, tris=None):
    """c * pull-back of per-triangle derivatives to the vertices -> grad [nv,3]."""
    lib = _load()
    V, F = _prep(V, F)
    grad = np.zeros_like(V)
    gw = np.ascontiguousarray(gw, dtype=np.float64)
    gnu = np.ascontiguousarray(gnu, dtype=np.float64)
    gx = np.ascontiguousarray(gx, dtype=np.float64)
    if tris is None:
        lib.or_adjoint(V, F, None, F.shape[0], gw, gnu, gx, c, grad)
    else:
        lst = np.ascontiguousarray(tris, dtype=np.int64)
        lib.or_adjoint(V, F, lst.ctypes.data_as(C.c_void_p), lst.shape[0], gw, gnu, gx, c, grad)
    return grad


def gradient(V, F, q=6.0, p=12.0, c=1.0, adj=0, nthreads=None):
    """(Phi, dPhi/dV [nv,3]) by the exact chain rule; Phi = c/2 sum_T w_T dPhi/dw_T is NOT used:
    the energy is the plain double sum."""
    x, nu, w = tri_data(V, F)
    E = energy_soa(x, nu, w, F, q, p, c, adj, nthreads)
    gw, gnu, gx = tri_accum(V, F, None, q, p, adj, nthreads, soa=(x, nu, w))
    return E, adjoint(V, F, gw, gnu, gx, c)


def incident_triangles(F, verts):
    """Triangles touching any of ``verts`` (sorted unique)."""
    F = np.asarray(F)
    mask = np.isin(F, np.asarray(verts)).any(axis=1)
    return np.nonzero(mask)[0].astype(np.int64)


def vertex_gradient_sample(V, F, verts, q=6.0, p=12.0, c=1.0, adj=0, nthreads=None):
    """Exact dPhi/dv for the listed vertices only (cost O(#incident * nt))."""
    tris = incident_triangles(F, verts)
    gw, gnu, gx = tri_accum(V, F, tris, q, p, adj, nthreads)
    grad = adjoint(V, F, gw, gnu, gx, c, tris=tris)
    return grad[np.asarray(verts)]


def lbvh(x, morton_bits=30, leaf_size=16):
    """Morton codes, sorted permutation and radix tree (see or_lbvh)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    nn = 2 * n - 1
    codes = np.zeros(n, dtype=np.uint32)
    perm = np.zeros(n, dtype=np.int32)
    left = np.full(max(n - 1, 1), -1, dtype=np.int32)
    right = np.full(max(n - 1, 1), -1, dtype=np.int32)
    parent = np.zeros(nn, dtype=np.int32)
    first = np.zeros(nn, dtype=np.int32)
    last = np.zeros(nn, dtype=np.int32)
    leaves = np.zeros(n, dtype=np.int32)
    nl = C.c_int64(0)
    rc = lib.or_lbvh(x, n, morton_bits, leaf_size, codes, perm, left, right, parent, first, last, leaves, C.byref(nl))
    if rc != 0:
        raise ValueError("or_lbvh: bad arguments")
    return dict(codes=codes, perm=perm, left=left[: n - 1], right=right[: n - 1], parent=parent,
                first=first, last=last, leaves=leaves[: nl.value].copy(), n=n, leaf_size=leaf_size)


def moments(V, F, tree, soa=None):
    """Per-node moments [2n-1,13] (A, wX, wnu, wnu(x)nu upper) and vertex boxes [2n-1,6]."""
    lib = _load()
    V, F = _prep(V, F)
    x, nu, w = soa if soa is not None else tri_data(V, F)
    n = tree["n"]
    mom = np.zeros((2 * n - 1, 13))
    box = np.zeros((2 * n - 1, 6))
    left = np.ascontiguousarray(np.concatenate([tree["left"], [-1]]).astype(np.int32))
    right = np.ascontiguousarray(np.concatenate([tree["right"], [-1]]).astype(np.int32))
    lib.or_moments(V, F, x, nu, w, n, tree["perm"], left, right, mom, box)
    return mom, box


def bh_accum(V, F, tree, mom, box, theta, q=6.0, p=12.0, adj=0, nthreads=None, soa=None):
    """Barnes-Hut per-triangle derivatives (without c) and (#near pairs, #far terms)."""
    lib = _load()
    V, F = _prep(V, F)
    x, nu, w = soa if soa is not None else tri_data(V, F)
    n = tree["n"]
    gw = np.zeros(n)
    gnu = np.zeros((n, 3))
    gx = np.zeros((n, 3))
    nn, nf = C.c_int64(0), C.c_int64(0)
    left = np.ascontiguousarray(np.concatenate([tree["left"], [-1]]).astype(np.int32))
    right = np.ascontiguousarray(np.concatenate([tree["right"], [-1]]).astype(np.int32))
    lib.or_bh_accum(x, nu, w, F, n, tree["perm"], left, right, tree["first"], tree["last"],
                    tree["leaves"], tree["leaves"].shape[0], np.ascontiguousarray(mom), np.ascontiguousarray(box),
                    theta, tree["leaf_size"], q, p, adj, gw, gnu, gx, C.byref(nn), C.byref(nf),
                    nthreads or nthreads_default())
    return gw, gnu, gx, nn.value, nf.value


def bh_gradient(V, F, theta, q=6.0, p=12.0, c=1.0, adj=0, morton_bits=30, leaf_size=16, nthreads=None):
    """(Phi_BH, grad_BH, info): Phi_BH = c/2 sum_T w_T dPhi/dw_T over both orderings."""
    x, nu, w = tri_data(V, F)
    tree = lbvh(x, morton_bits, leaf_size)
    mom, box = moments(V, F, tree, soa=(x, nu, w))
    gw, gnu, gx, nn, nf = bh_accum(V, F, tree, mom, box, theta, q, p, adj, nthreads, soa=(x, nu, w))
    E = 0.5 * c * float(np.sum(w * gw))
    grad = adjoint(V, F, gw, gnu, gx, c)
    return E, grad, dict(near_pairs=nn, far_terms=nf, tree=tree, mom=mom, box=box, gw=gw, gnu=gnu, gx=gx)


# ---------------------------------------------------------------- learned far field
MLP_NI, MLP_NH, MLP_NO = 24, 64, 7


def dt_accum(V, F, tree, mom, box, theta, q=6.0, p=12.0, adj=0, soa=None):
    """Cluster-cluster (dual-tree) Barnes-Hut form (see or_dt_accum): per-triangle
    derivatives (without c), the energy (without c) and the pair counts."""
    lib = _load()
    V, F = _prep(V, F)
    x, nu, w = soa if soa is not None else tri_data(V, F)
    n = tree["n"]
    gw = np.zeros(n)
    gnu = np.zeros((n, 3))
    gx = np.zeros((n, 3))
    nn, nf, nr = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    left = np.ascontiguousarray(np.concatenate([tree["left"], [-1]]).astype(np.int32))
    right = np.ascontiguousarray(np.concatenate([tree["right"], [-1]]).astype(np.int32))
    E = lib.or_dt_accum(np.ascontiguousarray(x), np.ascontiguousarray(nu), np.ascontiguousarray(w), F, n,
                        tree["perm"], left, right, tree["parent"], tree["first"], tree["last"],
                        np.ascontiguousarray(mom), np.ascontiguousarray(box), theta, tree["leaf_size"], q, p, adj,
                        gw, gnu, gx, C.byref(nn), C.byref(nf), C.byref(nr))
    return E, gw, gnu, gx, {"near_pairs": nn.value, "far_pairs": nf.value, "far_represented": nr.value}


def dt_gradient(V, F, theta, q=6.0, p=12.0, c=1.0, adj=0, morton_bits=30, leaf_size=16):
    """(Phi_DT, grad_DT, info) of the cluster-cluster form with prefactor c."""
    x, nu, w = tri_data(V, F)
    tree = lbvh(x, morton_bits, leaf_size)
    mom, box = moments(V, F, tree, soa=(x, nu, w))
    E, gw, gnu, gx, info = dt_accum(V, F, tree, mom, box, theta, q, p, adj, soa=(x, nu, w))
    grad = adjoint(V, F, gw, gnu, gx, c)
    info["phi_from_weights"] = 0.5 * c * float(np.sum(w * gw))
    return c * E, grad, info


def mlp_nparam():
    return int(_load().or_mlp_nparam())


def mlp_forward(params, X):
    """Network outputs [n,7] for normalised inputs X [n,24] (FP64)."""
    lib = _load()
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.zeros((X.shape[0], MLP_NO))
    lib.or_mlp_forward(P, X.shape[0], X, Y)
    return Y


def mlp_loss_grad(params, X, T, M):
    """(loss, dL/dparams) of the masked mean-square loss."""
    lib = _load()
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    Y = mlp_forward(P, X)
    dY = np.zeros_like(Y)
    L = lib.or_mlp_loss(X.shape[0], Y, T, M, dY.ctypes.data_as(C.c_void_p))
    dP = np.zeros_like(P)
    lib.or_mlp_backward(P, X.shape[0], X, dY, dP)
    return L, dP


def adamw_step(w, m, v, g, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0, t=1):
    """In-place AdamW step on FP64 arrays."""
    lib = _load()
    for a in (w, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib.or_adamw_step(w, m, v, g, w.size, lr, b1, b2, eps, wd, t)


def far_features(momL, boxL, momC, boxC):
    lib = _load()
    f = np.zeros(MLP_NI)
    lib.or_far_features(*(np.ascontiguousarray(a, dtype=np.float64) for a in (momL, boxL, momC, boxC)), f)
    return f


def far_channels(x, nu, w, targets, members, momC, q=6.0, p=12.0):
    """(monopole[7], exact[7]) channel sums of one (leaf, cluster) pair."""
    lib = _load()
    tl = np.ascontiguousarray(targets, dtype=np.int64)
    sc = np.ascontiguousarray(members, dtype=np.int64)
    mono = np.zeros(7)
    exact = np.zeros(7)
    lib.or_far_channels(np.ascontiguousarray(x, dtype=np.float64), np.ascontiguousarray(nu, dtype=np.float64),
                        np.ascontiguousarray(w, dtype=np.float64), tl, tl.size, sc, sc.size,
                        np.ascontiguousarray(momC, dtype=np.float64), q, p, mono, exact)
    return mono, exact


# ---------------------------------------------------------------- confinement (Eq. TPConf)
def conf_data(Vc, Fc):
    """Centroids y [nk,3] and areas a [nk] of the confining surface's triangles."""
    y, _, a = tri_data(Vc, Fc)
    return y, a


def conf_energy(V, F, Vc, Fc, q=6.0, p=12.0, c=1.0, soa=None, conf=None, nthreads=None):
    """Phi_conf = c sum_T sum_K w_T a_K |nu_T.(x_T - y_K)|^q / |x_T - y_K|^p (Eq. TPConf)."""
    lib = _load()
    x, nu, w = soa if soa is not None else tri_data(V, F)
    y, a = conf if conf is not None else conf_data(Vc, Fc)
    x, nu, w, y, a = (np.ascontiguousarray(t, dtype=np.float64) for t in (x, nu, w, y, a))
    return lib.or_conf_energy(x, nu, w, x.shape[0], y, a, y.shape[0], q, p, c, nthreads or nthreads_default())


def conf_accum(V, F, Vc, Fc, q=6.0, p=12.0, soa=None, conf=None, nthreads=None):
    """Per-triangle dPhi_conf/dw_T, dPhi_conf/dnu_T [.,3], dPhi_conf/dx_T [.,3] (without c)."""
    lib = _load()
    x, nu, w = soa if soa is not None else tri_data(V, F)
    y, a = conf if conf is not None else conf_data(Vc, Fc)
    x, nu, w, y, a = (np.ascontiguousarray(t, dtype=np.float64) for t in (x, nu, w, y, a))
    nt = x.shape[0]
    gw, gnu, gx = np.zeros(nt), np.zeros((nt, 3)), np.zeros((nt, 3))
    lib.or_conf_accum(x, nu, w, nt, y, a, y.shape[0], q, p, gw, gnu, gx, nthreads or nthreads_default())
    return gw, gnu, gx


def conf_gradient(V, F, Vc, Fc, q=6.0, p=12.0, c=1.0, nthreads=None):
    """(Phi_conf, dPhi_conf/dV [nv,3]): only the evolving surface moves."""
    x, nu, w = tri_data(V, F)
    conf = conf_data(Vc, Fc)
    E = conf_energy(V, F, Vc, Fc, q, p, c, soa=(x, nu, w), conf=conf, nthreads=nthreads)
    gw, gnu, gx = conf_accum(V, F, Vc, Fc, q, p, soa=(x, nu, w), conf=conf, nthreads=nthreads)
    return E, adjoint(V, F, gw, gnu, gx, c)


def conf_vertex_gradient_sample(V, F, Vc, Fc, verts, q=6.0, p=12.0, c=1.0, nthreads=None):
    """Exact dPhi_conf/dv for the listed vertices of the evolving surface only."""
    tris = incident_triangles(F, verts)
    x, nu, w = tri_data(V, F)
    gw, gnu, gx = conf_accum(V, F, Vc, Fc, q, p, soa=(x[tris], nu[tris], w[tris]), nthreads=nthreads)
    grad = adjoint(V, F, gw, gnu, gx, c, tris=tris)
    return grad[np.asarray(verts)]


# ---------------------------------------------------------------- multi-point quadrature (Sec. 3.1, 3.2)
def quad_rule(k):
    """Symmetric triangle rules with barycentric points [k,3] and weights [k] (sum 1):
    k = 1 the centroid (degree 1), k = 3 the points (2/3, 1/6, 1/6) (degree 2), k = 6 the
    degree-4 rule of Strang and Fix (closed forms of its two orbits)."""
    if k == 1:
        return np.array([[1 / 3, 1 / 3, 1 / 3]]), np.array([1.0])
    if k == 3:
        a, b = 2.0 / 3.0, 1.0 / 6.0
        return np.array([[a, b, b], [b, a, b], [b, b, a]]), np.full(3, 1.0 / 3.0)
    if k == 6:
        s10, r = np.sqrt(10.0), np.sqrt(38.0 - 44.0 * np.sqrt(2.0 / 5.0))
        a1, a2 = (8.0 - s10 + r) / 18.0, (8.0 - s10 - r) / 18.0
        t = np.sqrt(213125.0 - 53320.0 * s10)
        w1, w2 = (620.0 + t) / 3720.0, (620.0 - t) / 3720.0
        pts, wts = [], []
        for a, w in ((a1, w1), (a2, w2)):
            c = 1.0 - 2.0 * a
            pts += [[c, a, a], [a, c, a], [a, a, c]]
            wts += [w, w, w]
        return np.array(pts), np.array(wts)
    raise ValueError("quadrature with 1, 3 or 6 points")


def quad_points(V, F, k):
    """Quadrature points of every triangle: x [nt*k,3], nu, w [nt*k], parent faces [nt*k,3]."""
    lib = _load()
    V, F = _prep(V, F)
    bary, om = quad_rule(k)
    bary = np.ascontiguousarray(bary, dtype=np.float64)
    om = np.ascontiguousarray(om, dtype=np.float64)
    n = F.shape[0] * k
    x, nu, w = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    Fq = np.zeros((n, 3), dtype=np.int32)
    lib.or_quad_points(V, F, F.shape[0], k, bary, om, x, nu, w, Fq)
    return x, nu, w, Fq


def quad_energy(V, F, k, q=6.0, p=12.0, c=1.0, nthreads=None):
    """Phi with k quadrature points per triangle on both integrals (pairs of points of admitted triangles)."""
    x, nu, w, Fq = quad_points(V, F, k)
    return energy_soa(x, nu, w, Fq, q, p, c, 0, nthreads)


def quad_gradient(V, F, k, q=6.0, p=12.0, c=1.0, nthreads=None):
    """(Phi, dPhi/dV) of the k-point quadrature form."""
    lib = _load()
    V, F = _prep(V, F)
    x, nu, w, Fq = quad_points(V, F, k)
    E = energy_soa(x, nu, w, Fq, q, p, c, 0, nthreads)
    gw, gnu, gx = tri_accum(V, Fq, None, q, p, 0, nthreads, soa=(x, nu, w))
    bary, om = quad_rule(k)
    grad = np.zeros_like(V)
    lib.or_quad_adjoint(V, F, F.shape[0], k, np.ascontiguousarray(bary), np.ascontiguousarray(om),
                        np.ascontiguousarray(gw), np.ascontiguousarray(gnu), np.ascontiguousarray(gx), c, grad)
    return E, grad
