"""CPU emulation of the tile schedule of the fused iteration, against Algorithm 5.

The GPU path splits one iteration of Algorithm 5 over tiles of cells: every
tile recomputes the "pre" values (r_k, p_k) of all nodes of its node brick from
the previous iteration's buffers, while only the owner of a node stores them;
it applies the operator to its own cells into the brick; nodes whose every
contribution lies inside the tile are finished there (v_k stored, the seven
sums accumulated, Dirichlet rows as identity), and nodes on faces shared with
another tile leave a partial sum in the shell buffer, which the tail adds up
in a fixed order before it accumulates their sums.  This module restates that
schedule in numpy (ownership by i // (p T) capped at the last tile, lower-face
partials, "+"-face partials, the tail) and checks that it reproduces the
oracle's Algorithm 5 on the assembled matrix: the same alpha_k and beta_k, the
same iterate, every node's r_k, p_k and v_k stored exactly once.
"""
import itertools

import numpy as np
import pytest

from oracle import cg, fem


def _owner(i, p, T, nt):
    return min(i // (p * T), nt - 1)


class TileSchedule:
    def __init__(self, prob, T):
        self.prob, self.T = prob, T
        p = prob.p
        N = prob.cells
        self.nn = prob.nodes_per_dim
        self.nt = tuple(-(-N[d] // T[d]) for d in range(3))
        self.gid = fem.local_to_global(prob)
        if fem.cartesian_cells_identical(prob):
            self.Ae = np.broadcast_to(fem.element_matrices(prob, np.array([0]))[0],
                                      (prob.n_cells,) + (self.gid.shape[1],) * 2)
        else:
            self.Ae = fem.element_matrices(prob)
        self.dirichlet = fem.boundary_mask(prob)
        nx, ny, _ = self.nn
        self.tiles = []
        for tz, ty, tx in itertools.product(range(self.nt[2]), range(self.nt[1]), range(self.nt[0])):
            t = (tx, ty, tz)
            c0 = [t[d] * T[d] for d in range(3)]
            nc = [min(T[d], N[d] - c0[d]) for d in range(3)]
            rng = [np.arange(p * c0[d], p * (c0[d] + nc[d]) + 1) for d in range(3)]
            K, J, I = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
            I, J, K = I.ravel(), J.ravel(), K.ravel()
            ids = I + nx * (J + ny * K)
            own = np.array([_owner(i, p, T[0], self.nt[0]) == tx and _owner(j, p, T[1], self.nt[1]) == ty
                            and _owner(k, p, T[2], self.nt[2]) == tz for i, j, k in zip(I, J, K)])
            # owned nodes on a lower face shared with the previous tile
            lower = ((I == p * c0[0]) & (tx > 0)) | ((J == p * c0[1]) & (ty > 0)) | ((K == p * c0[2]) & (tz > 0))
            cells = [cx + N[0] * (cy + N[1] * cz) for cz in range(c0[2], c0[2] + nc[2])
                     for cy in range(c0[1], c0[1] + nc[1]) for cx in range(c0[0], c0[0] + nc[0])]
            self.tiles.append(dict(ids=ids, own=own, lower=lower, cells=np.array(cells)))

    def iterate(self, b, dinv, K):
        """K fused iterations from x0 = 0; returns (alphas, betas, x, store counts)."""
        n = self.prob.n_dofs
        dirichlet = self.dirichlet
        r_o, p_o, v_o, x = b.copy(), np.zeros(n), np.zeros(n), np.zeros(n)
        al = {0: 0.0, -1: 0.0}
        be = {0: 0.0, -1: 0.0}
        alphas, betas = [], []
        counts = []
        for k in range(1, K + 1):
            r_n, p_n, v_n = np.full(n, np.nan), np.full(n, np.nan), np.full(n, np.nan)
            stores = np.zeros((3, n), dtype=int)
            sums = np.zeros(7)
            shell = []  # (tile index, global ids, partial values)
            for ti, tl in enumerate(self.tiles):
                ids, own = tl["ids"], tl["own"]
                # phase 1: pre on every brick node from the previous buffers
                rk = r_o[ids] - al[k - 1] * v_o[ids]
                pk = dinv[ids] * rk + be[k - 1] * p_o[ids]
                U = np.where(dirichlet[ids], 0.0, pk)
                r_n[ids[own]] = rk[own]
                p_n[ids[own]] = pk[own]
                stores[0, ids[own]] += 1
                stores[1, ids[own]] += 1
                if k > 1 and k % 2 == 1:
                    o = ids[own]
                    x[o] += al[k - 1] * p_o[o] + (al[k - 2] / be[k - 2]) * (p_o[o] - dinv[o] * r_o[o])
                # phase 2: the tile's cells into the brick
                loc = {g: m for m, g in enumerate(ids)}
                V = np.zeros(len(ids))
                for c in tl["cells"]:
                    lc = np.array([loc[g] for g in self.gid[c]])
                    V[lc] += self.Ae[c] @ U[lc]
                # phase 3: finished owned nodes, shell partials for shared ones
                dirt = dirichlet[ids]
                shared = ~dirt & (~own | tl["lower"])
                fin = own & ~shared
                v = np.where(dirt, pk, V)
                f = ids[fin]
                v_n[f] = v[fin]
                stores[2, f] += 1
                sums += _post(rk[fin], pk[fin], v[fin], dinv[f])
                shell.append((ti, ids[shared], V[shared]))
            # tail: the partials of every shared node, in tile order
            acc, seen = {}, {}
            for ti, g_ids, vals in shell:
                for g, val in zip(g_ids, vals):
                    acc[g] = acc.get(g, 0.0) + val
                    seen[g] = seen.get(g, 0) + 1
            tail = np.array(sorted(acc))
            if len(tail):
                vt = np.array([acc[g] for g in tail])
                v_n[tail] = vt
                stores[2, tail] += 1
                sums += _post(r_n[tail], p_n[tail], vt, dinv[tail])
            counts.append((stores, seen))
            # reduction and the scalar step (Eqs. 7-8)
            g_, a_, b_, c_, d_, e_, f_ = sums
            al[k] = d_ / a_
            alphas.append(al[k])
            be[k] = (d_ - 2 * al[k] * e_ + al[k] ** 2 * f_) / d_
            betas.append(be[k])
            r_o, p_o, v_o = r_n, p_n, v_n
        # finalisation by the parity of K (Algorithm 5)
        if K % 2 == 1:
            x = x + al[K] * p_o
        else:
            x = x + al[K] * p_o + (al[K - 1] / be[K - 1]) * (p_o - dinv * r_o)
        return alphas, betas, x, counts


def _post(r, p, v, d):
    return np.array([r @ r, p @ v, r @ v, v @ v, r @ (d * r), r @ (d * v), v @ (d * v)])


@pytest.mark.parametrize("p,cells,T,amp", [(2, (5, 4, 3), (2, 2, 2), 0.0), (3, (4, 3, 5), (2, 3, 2), 0.05),
                                           (1, (6, 5, 4), (4, 2, 3), 0.0)])
def test_tile_schedule_reproduces_algorithm5(p, cells, T, amp):
    prob = fem.Problem(p=p, cells=cells, amplitude=amp)
    A = fem.assemble(prob)
    dinv = 1.0 / fem.diagonal(A)
    rng = np.random.default_rng(220508909 + 17 * p)
    b = rng.standard_normal(prob.n_dofs)
    b[fem.boundary_mask(prob)] = 0.0
    K = 7  # odd and even iterations, several delayed x updates
    sched = TileSchedule(prob, T)
    alphas, betas, x, counts = sched.iterate(b, dinv, K)
    ref = cg.pcg_algorithm5(lambda u: A @ u, b, dinv, 0.0, K)
    np.testing.assert_allclose(alphas, ref.alphas[:K], rtol=1e-11)
    np.testing.assert_allclose(betas[:K - 1], ref.betas[:K - 1], rtol=1e-10)
    np.testing.assert_allclose(x, ref.x, rtol=0, atol=1e-11 * np.abs(ref.x).max())
    for stores, seen in counts:
        # every node's r_k, p_k and v_k are stored exactly once
        assert (stores == 1).all()
        # shared nodes collect one partial per tile whose brick holds them: 2, 4 or 8
        assert set(seen.values()) <= {2, 4, 8}
