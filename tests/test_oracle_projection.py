"""Pins of the oracle's compatibility projection (Sec. 3.5) against an independent assembly.

The projection fits displacements u^c on the active-node graph to the deformation gradient: every
pair of active axis neighbours (m, l) asks u_m - u_l = 1/2 (G_m + G_l)(X_m - X_l) (G = F - I, Eq.
projection-edge-relation), every velocity-Dirichlet cut link of m asks u_m = u_D(X_b) + G_m (X_m -
X_b) (boundary edges), and the least-squares solution satisfies the graph-Laplacian normal
equations deg_m u_m - sum_l u_l = sum_l g_ml + sum_links b.  The oracle iterates damped Jacobi
sweeps toward it (a fixed count per solve in the method; here enough sweeps to converge), and with
no Dirichlet link fixes the free constant by a zero mean shift.  The test assembles the same system
from the geometry alone with scipy, solves it directly and compares; then checks F^c = I + grad u^c
(central differences where both axis neighbours are active, one-sided otherwise; Eq.
projection-compatible-F) against the oracle's.
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from paper_2606_20646_b300 import inputs as I


def _smooth_G(p, amp=0.05, seed=4):
    """A smooth, incompatible field G = F - I (low Fourier modes), (D*D, *box)."""
    rng = np.random.default_rng(seed)
    X = p.coords()
    D = p.dim
    G = np.zeros((D * D,) + p.box_shape)
    for k in range(D * D):
        ph = rng.uniform(0, 2 * np.pi, size=D)
        w = rng.integers(1, 3, size=D)
        G[k] = amp * np.prod([np.cos(np.pi * w[a] * X[a] + ph[a]) for a in range(D)], axis=0)
    return G


def _neighbour(p, idx, A, s):
    """Box index of the axis neighbour (no periodic boxes here), or None outside the box."""
    j = list(idx)
    j[A] += s
    if not (0 <= j[A] < p.n[A]):
        return None
    return tuple(j)


def _assemble(p, act, G, links, dirichlet_zero):
    """Normal equations of the projection's least-squares problem, one component at a time."""
    D, dx = p.dim, p.dx
    shape = p.box_shape                      # (nz, ny, nx) or (ny, nx): last axis is x
    nodes = [tuple(i) for i in np.argwhere(act)]
    num = {nd: i for i, nd in enumerate(nodes)}
    n = len(nodes)
    axis_of = lambda A: len(shape) - 1 - A   # array axis of lattice direction A
    rows, cols, vals = [], [], []
    rhs = np.zeros((D, n))
    deg = np.zeros(n)
    for i, nd in enumerate(nodes):
        for A in range(D):
            for s in (1, -1):
                nb = _neighbour(p, nd, axis_of(A), s)
                if nb is None or not act[nb]:
                    continue
                j = num[nb]
                deg[i] += 1.0
                rows.append(i)
                cols.append(j)
                vals.append(-1.0)
                for c in range(D):
                    Gm = G[(c * D + A,) + nd]
                    Gl = G[(c * D + A,) + nb]
                    rhs[c, i] += 0.5 * (Gm + Gl) * (-s * dx)       # X_m - X_l = -s dx e_A
    flat_to_idx = lambda m: np.unravel_index(m, shape)
    for m, q, eta in zip(links["node"], links["q"], links["eta"]):
        nd = tuple(int(v) for v in flat_to_idx(int(m)))
        i = num[nd]
        A, s = q // 2, (1.0 if q % 2 == 0 else -1.0)
        deg[i] += 1.0
        assert dirichlet_zero
        for c in range(D):
            rhs[c, i] += G[(c * D + A,) + nd] * (-s * eta * dx)    # X_m - X_b = -eta dx e
    Lap = sp.csr_matrix((vals, (rows, cols)), shape=(n, n)) + sp.diags(deg)
    return nodes, Lap, rhs


def _oracle_projection(p, G, sweeps):
    D = p.dim
    q = p.with_(options=dataclasses.replace(p.options, proj_iters=sweeps))
    o = oracle.Oracle(q).set_initial()
    eye = np.eye(D).reshape((D * D,) + (1,) * D)
    uc, Fc = o.project(G + eye, np.zeros((D,) + p.box_shape))
    act = o.active_mask().reshape(p.box_shape).astype(bool)
    return o, uc, Fc, act


def _check_compatible_F(p, act, uc, Fc, G):
    D, dx = p.dim, p.dx
    shape = p.box_shape
    axis_of = lambda A: len(shape) - 1 - A
    for nd in [tuple(i) for i in np.argwhere(act)]:
        for A in range(D):
            npos = _neighbour(p, nd, axis_of(A), 1)
            nneg = _neighbour(p, nd, axis_of(A), -1)
            ap = npos is not None and act[npos]
            am = nneg is not None and act[nneg]
            for c in range(D):
                if ap and am:
                    g = (uc[(c,) + npos] - uc[(c,) + nneg]) / (2 * dx)
                elif ap:
                    g = (uc[(c,) + npos] - uc[(c,) + nd]) / dx
                elif am:
                    g = (uc[(c,) + nd] - uc[(c,) + nneg]) / dx
                else:
                    g = G[(c * D + A,) + nd]          # keeps F
                want = (1.0 if c == A else 0.0) + g
                assert abs(Fc[(c * D + A,) + nd] - want) < 1e-12


def test_projection_with_dirichlet_anchors_solves_the_normal_equations():
    """Clamped cube (every face link velocity-Dirichlet zero, eta = 0.2): a nonsingular system."""
    p = I.inclusion_cube(6, 1)
    G = _smooth_G(p)
    o, uc, Fc, act = _oracle_projection(p, G, 4000)
    nodes, Lap, rhs = _assemble(p, act, G, o.links(), dirichlet_zero=True)
    for c in range(p.dim):
        x = spla.spsolve(Lap.tocsc(), rhs[c])
        got = np.array([uc[(c,) + nd] for nd in nodes])
        assert np.abs(got - x).max() <= 1e-12 * max(1.0, np.abs(x).max()), c
    assert not (~act).any() or np.abs(uc[:, ~act]).max() == 0.0
    _check_compatible_F(p, act, uc, Fc, G)


def test_projection_without_anchors_is_the_zero_mean_solution():
    """Periodic-free body with only Neumann links (the thick shell): the normal equations fix u^c up
    to a constant; the oracle's gauge makes its mean zero (warm start 0)."""
    p = I.shell_3d(12)
    G = _smooth_G(p, amp=0.03, seed=9)
    o, uc, Fc, act = _oracle_projection(p, G, 6000)
    links = o.links()
    nodes, Lap, rhs = _assemble(p, act, G, {"node": [], "q": [], "eta": []}, dirichlet_zero=True)
    n = len(nodes)
    for c in range(p.dim):
        # pin the constant by the zero mean: solve [Lap 1; 1^T 0] [x; k] = [rhs; 0]
        ones = np.ones((n, 1))
        M = sp.bmat([[Lap, sp.csr_matrix(ones)], [sp.csr_matrix(ones.T), None]]).tocsc()
        x = spla.spsolve(M, np.concatenate([rhs[c], [0.0]]))[:n]
        got = np.array([uc[(c,) + nd] for nd in nodes])
        assert abs(got.mean()) < 1e-12
        assert np.abs(got - x).max() <= 1e-9 * max(1.0, np.abs(x).max()), (c, np.abs(got - x).max())
    assert len(links["node"]) > 0 and o.counts()["n_dirichlet"] == 0
    _check_compatible_F(p, act, uc, Fc, G)
