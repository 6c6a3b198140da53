"""FP64 oracle of the elastic term of the quasi-static simulation (test infrastructure only).

The paper shows a quasi-static simulation with its energy that evolves from an invalid
state to a valid one (Fig. 2) but does not state the elastic model.  The reading used
here is a mass-spring term, plus optional anchors:

  E_el(x) = sum over springs (i, j) of k/2 (|x_i - x_j| - L_ij)^2
          + sum over anchors v of k_a/2 |x_v - t_v|^2

and the simulation minimises E_el + sum T with the same inexact Newton iteration as the
plain solve, stopping when no pair intersects.  Every function below is the definition
written out: the spring's exact 6x6 Hessian from its analytic form, then the nearest PSD
matrix by clamping negative eigenvalues (numpy eigh), scattered into 3x3 vertex blocks.

Parity status: pinned (tests/test_oracle.py): zero energy and gradient at rest, a
stretched spring's closed form, central finite differences of the energy (gradient) and
of the gradient (unprojected Hessian), the closed-form spectrum of the projected spring
Hessian {2k, 2k max(0, 1 - L/l) (twice), 0 (three times)}, translation and rotation
invariance of the spring energy.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .ttie_oracle import (NewtonParams, assemble, blocks_to_dense, candidate_pairs,
                          capped_direction, clamp_psd, evaluate, line_search, next_overshoot, pair_dofs)


@dataclass
class Elastic:
    edges: np.ndarray                 # [E,2] vertex ids of the springs
    rest: np.ndarray                  # [E] rest lengths
    k_edge: float = 1.0
    anchors: np.ndarray | None = None  # [A] vertex ids held by zero-length springs
    targets: np.ndarray | None = None  # [A,3] their anchor points
    k_anchor: float = 0.0

    def n_anchors(self) -> int:
        return 0 if self.anchors is None else len(self.anchors)


def mesh_edges(tri: np.ndarray) -> np.ndarray:
    """Unique undirected edges (i < j) of a triangle mesh, sorted."""
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def springs_at_rest(x: np.ndarray, tri: np.ndarray, k_edge: float) -> Elastic:
    """Springs on every mesh edge with the current lengths as rest lengths."""
    e = mesh_edges(tri)
    return Elastic(e, np.linalg.norm(x[e[:, 0]] - x[e[:, 1]], axis=1), k_edge)


def elastic_energy(x: np.ndarray, el: Elastic) -> float:
    d = x[el.edges[:, 0]] - x[el.edges[:, 1]]
    l = np.linalg.norm(d, axis=1)
    E = 0.5 * el.k_edge * float(np.sum((l - el.rest) ** 2))
    if el.n_anchors():
        E += 0.5 * el.k_anchor * float(np.sum((x[el.anchors] - el.targets) ** 2))
    return E


def elastic_gradient(x: np.ndarray, el: Elastic) -> np.ndarray:
    """[V,3]: k (l - L) (x_i - x_j)/l on i, the negative on j; k_a (x_v - t_v) on anchors."""
    g = np.zeros_like(x, dtype=np.float64)
    d = x[el.edges[:, 0]] - x[el.edges[:, 1]]
    l = np.linalg.norm(d, axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        f = np.where(l > 0, el.k_edge * (l - el.rest) / l, 0.0)
    np.add.at(g, el.edges[:, 0], f[:, None] * d)
    np.add.at(g, el.edges[:, 1], -f[:, None] * d)
    if el.n_anchors():
        np.add.at(g, el.anchors, el.k_anchor * (x[el.anchors] - el.targets))
    return g


def spring_hessian(xi: np.ndarray, xj: np.ndarray, L: float, k: float) -> np.ndarray:
    """Exact 6x6 Hessian of k/2 (|xi - xj| - L)^2 over (xi, xj): [[K, -K], [-K, K]] with
    K = k (n n' + (1 - L/l)(I - n n')), n = (xi - xj)/l.  A zero-length spring (l = 0) has
    no direction: K = k I there (the limit of the stretched case along any n)."""
    d = np.asarray(xi, np.float64) - np.asarray(xj, np.float64)
    l = float(np.linalg.norm(d))
    if l == 0.0:
        K = k * np.eye(3)
    else:
        n = d / l
        P = np.outer(n, n)
        K = k * (P + (1.0 - L / l) * (np.eye(3) - P))
    return np.block([[K, -K], [-K, K]])


def elastic_blocks(x: np.ndarray, el: Elastic, psd: bool = True) -> dict:
    """{(row_vertex, col_vertex): 3x3}: every spring's 6x6 Hessian (projected to PSD by
    clamping its negative eigenvalues when psd) and k_a I on every anchor."""
    blocks: dict = {}

    def add(key, b):
        blocks[key] = blocks[key] + b if key in blocks else b.copy()

    for (i, j), L in zip(el.edges, el.rest):
        H = spring_hessian(x[i], x[j], float(L), el.k_edge)
        if psd:
            H = clamp_psd(H[None])[0]
        v = (int(i), int(j))
        for r in range(2):
            for c in range(2):
                add((v[r], v[c]), H[3 * r:3 * r + 3, 3 * c:3 * c + 3])
    if el.n_anchors():
        for a in el.anchors:
            add((int(a), int(a)), el.k_anchor * np.eye(3))
    return blocks


def elastic_vertices(el: Elastic) -> np.ndarray:
    v = [el.edges.ravel()]
    if el.n_anchors():
        v.append(np.asarray(el.anchors).ravel())
    return np.unique(np.concatenate(v))


def total_energy(x, tri, group, prm: NewtonParams, el: Elastic):
    """(E_el + sum T, intersecting pairs) at x."""
    pairs = candidate_pairs(x, tri, group, prm.mode)
    ev = evaluate(x, tri, pairs, prm.tc_scale)
    return float(ev.T.sum()) + elastic_energy(x, el), int(ev.active.sum())


def newton_direction_elastic(x, tri, group, prm: NewtonParams, el: Elastic):
    """One Newton system of E_el + sum T at x: returns (E, n_active, grad [V,3], d [V,3],
    rows).  The rows are the vertices of intersecting pairs, springs and anchors; H+ is
    the PSD Hessian of both terms; mu = mu_rel times its mean diagonal; d solves
    (H+ + mu I) d = -g on the rows.  With no intersecting pair the state is valid and d = 0."""
    V = x.shape[0]
    pairs = candidate_pairs(x, tri, group, prm.mode)
    ev = evaluate(x, tri, pairs, prm.tc_scale)
    n_act = int(ev.active.sum())
    E = float(ev.T.sum()) + elastic_energy(x, el)
    grad, blocks = assemble(tri, ev, V, prm.psd)
    grad = grad + elastic_gradient(x, el)
    d = np.zeros((V, 3))
    if n_act == 0:
        return E, 0, grad, d, np.zeros(0, np.int64)
    for key, b in elastic_blocks(x, el).items():
        blocks[key] = blocks[key] + b if key in blocks else b
    rows = np.unique(np.concatenate([pair_dofs(tri, ev.pairs[ev.active]).ravel(), elastic_vertices(el)]))
    H = blocks_to_dense(blocks, rows)
    mu = prm.mu_rel * float(np.mean(np.diag(H)))
    sol = np.linalg.solve(H + mu * np.eye(H.shape[0]), -grad[rows].ravel())
    d[rows] = sol.reshape(-1, 3)
    return E, n_act, grad, d, rows


def quasi_static_solve(x0, tri, group, prm: NewtonParams, el: Elastic, log=None):
    """The quasi-static simulation: inexact Newton on E_el + sum T with the plain solve's
    step cap, line search and overshoot (first trial 1 + eta, then 1, 1/2, ...; Armijo, no
    intersecting pair, or with rule "fewer" fewer pairs without raising E), from x0 until no
    pair intersects."""
    x = np.array(x0, dtype=np.float64)
    e = np.concatenate([x[tri[:, 1]] - x[tri[:, 0]], x[tri[:, 2]] - x[tri[:, 1]], x[tri[:, 0]] - x[tri[:, 2]]])
    cap = prm.max_step * float(np.linalg.norm(e, axis=1).mean())
    eta = prm.push_eta
    for it in range(prm.newton_max_it):
        E, n_act, grad, d, _ = newton_direction_elastic(x, tri, group, prm, el)
        if log is not None:
            log.append((it, E, n_act))
        if n_act == 0:
            return x, it, True
        d = capped_direction(d, cap)
        a, x, _, nt = line_search(x, d, E, float(np.sum(grad * d)),
                                  lambda xt: total_energy(xt, tri, group, prm, el), prm, n0=n_act, eta=eta)
        eta = next_overshoot(eta, a, n_act, nt, prm)
    return x, prm.newton_max_it, False
