"""Multigrid of Sec. 2.2 and the vertex-patch smoother of Sec. 2.3 / Sec. 3,
written with assembled matrices.

Transfer (Sec. 2.2): prolongation is the embedding V_{l-1} -> V_l, i.e.
P[i, J] = phi^{l-1}_J(x_i) for every active fine node i and active coarse
node J; restriction is P^T.

Patches (Sec. 2.3, covering reading): one per vertex X of an active cell; the
patch cells are the active cells around X; I_j are the patch's lattice nodes
all of whose active cells are patch cells (for a vertex whose 2^d cells are
active and uncut: the (2p-1)^d nodes strictly inside the patch), so that the
patches cover Omega_l; A_j = A_l[I_j, I_j].  The printed vertex set (mesh
vertices inside Omega, interior nodes only) leaves the DoFs near the boundary
in no patch; a test pins that consequence.

Smoother (eqs. "smoother", "smoother-split"), with these readings:
* the printed update drops y^{(j-1)} and flips the sign; the update used is
  y <- y + Q_j^T A_j^{-1} Q_j (b - A y);
* "interior" (Cartesian) patch: every patch cell is uncut and no face of a
  patch cell is a ghost face; every other patch is a cut patch;
* colour of the patch at vertex v: sum_k (v_k mod 2) 2^k;
* inconsistent ghost-penalty treatment (Sec. 2.3, last paragraph): within a
  colour one residual is formed and every patch of the colour is updated
  from it (additive within a colour, multiplicative across colours);
* pre-smoothing: interior colours 0..2^d-1, then n_c times the cut colours
  0..2^d-1; post-smoothing is the exact reverse sequence (this keeps the
  V-cycle symmetric, which CG needs).

V-cycle (Sec. 2.2): zero initial guess on every level, one pre- and one
post-smoothing step, exact solve on level 0.  Outer solver: CG preconditioned
by one V-cycle, x_0 = 0, stop at ||r||_2 <= rtol ||b||_2 on the recursive
residual.
"""

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .fem import Level, assemble_level, assemble_rhs


def prolongation_1d(basis, p, Nc):
    """Dense (p 2Nc + 1) x (p Nc + 1) matrix of coarse 1D nodal basis
    functions evaluated at the fine lattice nodes."""
    Nf = 2 * Nc
    nf, nc = p * Nf + 1, p * Nc + 1
    P = np.zeros((nf, nc))
    for I in range(nf):
        cf = min(I // p, Nf - 1)
        af = I - p * cf
        cc = cf // 2
        xi = ((cf % 2) + basis.nodes[af]) / 2.0
        vals = basis.eval(np.array([xi]))[:, 0]
        for a in range(p + 1):
            P[I, p * cc + a] += vals[a]
    return P


def prolongation(fine, coarse):
    P1 = sp.csr_matrix(prolongation_1d(fine.basis, fine.p, coarse.N))
    full = P1
    for _ in range(fine.d - 1):
        full = sp.kron(P1, full, format="csr")
    return full[fine.dof_nodes][:, coarse.dof_nodes].tocsr()


class Patches:
    """Vertex patches of one level with their colours and local matrices.

    Reading of Sec. 2.3: the patches must cover Omega_l, so there is one patch
    per vertex of an active cell; its cells are the active cells around the
    vertex; V_{l,j} is spanned by the basis functions whose support (within
    Omega_l) lies in the patch, i.e. I_j holds the patch nodes all of whose
    active cells are patch cells.  For a vertex whose 2^d cells are all active
    and uncut this is the (2p-1)^d interior nodes."""

    def __init__(self, lev, A):
        d, N, p = lev.d, lev.N, lev.p
        self.d = d
        act = np.zeros((N + 4,) * d, dtype=bool)       # padded, [c_{d-1}, .., c_0]
        cut = np.zeros((N + 4,) * d, dtype=bool)
        sl = tuple([slice(2, N + 2)] * d)
        act[sl] = lev.active.reshape((N,) * d)
        cut[sl] = lev.cut.reshape((N,) * d)

        def at(arr, v, delta):
            idx = tuple(v[:, k] + delta[k] + 2 for k in reversed(range(d)))
            return arr[idx]

        allv = np.array(np.meshgrid(*([np.arange(N + 1)] * d), indexing="ij")).reshape(d, -1).T
        cell_offs = np.array(np.meshgrid(*([np.array([-1, 0])] * d), indexing="ij")).reshape(d, -1).T
        any_act = np.zeros(allv.shape[0], dtype=bool)
        for dl in cell_offs:
            any_act |= at(act, allv, dl)
        verts = allv[any_act]
        self.verts = verts
        nv = verts.shape[0]
        # patch cells present / cut
        pc_act = np.stack([at(act, verts, dl) for dl in cell_offs], axis=1)
        pc_cut = np.stack([at(cut, verts, dl) for dl in cell_offs], axis=1)
        cart = pc_act.all(axis=1) & ~pc_cut.any(axis=1)
        for dl in cell_offs:
            for k in range(d):
                for s in (-1, 1):
                    nb = dl.copy()
                    nb[k] += s
                    cart &= ~at(cut, verts, nb)
        self.cut = ~cart
        # closure node offsets and the cells containing each
        c1 = 2 * p + 1
        node_offs = np.array(np.meshgrid(*([np.arange(c1)] * d), indexing="ij")).reshape(d, -1).T
        member = np.zeros((nv, node_offs.shape[0]), dtype=bool)
        for t, o in enumerate(node_offs):
            per_dim = []
            for k in range(d):
                ok = o[k]
                if ok == 0:
                    per_dim.append([-2, -1])
                elif ok < p:
                    per_dim.append([-1])
                elif ok == p:
                    per_dim.append([-1, 0])
                elif ok < 2 * p:
                    per_dim.append([0])
                else:
                    per_dim.append([0, 1])
            cells = np.array(np.meshgrid(*per_dim, indexing="ij")).reshape(d, -1).T
            inside_any = np.zeros(nv, dtype=bool)
            outside_any = np.zeros(nv, dtype=bool)
            for dl in cells:
                a = at(act, verts, dl)
                if ((dl == -1) | (dl == 0)).all():
                    inside_any |= a
                else:
                    outside_any |= a
            member[:, t] = inside_any & ~outside_any
        strides = lev.n ** np.arange(d)
        base = (p * (verts - 1)) @ strides
        off = node_offs @ strides
        self.I, self.Aj = [], []
        for j in range(nv):
            nodes = base[j] + off[member[j]]
            dofs = lev.node_to_dof[nodes]
            assert (dofs >= 0).all()
            self.I.append(dofs)
            Aj = A[dofs][:, dofs].toarray()
            self.Aj.append(Aj)
        self.colour = (verts % 2) @ (1 << np.arange(d))
        self.size = np.array([len(I) for I in self.I])

    def select(self, cut, colour):
        return np.nonzero((self.cut == cut) & (self.colour == colour))[0]


class LevelData:
    def __init__(self, ls, d, N, p, gamma_D, gammas, q):
        self.lev = Level(ls, d, N, p)
        self.A, self.parts = assemble_level(self.lev, gamma_D, gammas, q)
        self.patches = None


class Hierarchy:
    """Levels l = 0..L (N_l = N_L / 2^(L-l)), assembled operators, transfers,
    patches; V-cycle and PCG."""

    # Chebyshev smoother (the paper's comparison in Sec. 4): degree, power
    # iterations of the lambda_max estimate, safety factor, smoothing range
    CHEB_POWER_STEPS = 30
    CHEB_SAFETY = 1.2
    CHEB_RANGE = 20.0

    def __init__(self, ls, d, N, p, n_levels, gamma_D=None, gammas=None, q=None, n_c=2,
                 smoother="mvs", cheb_degree=5):
        self.d, self.p, self.n_c = d, p, n_c
        self.smoother, self.cheb_degree = smoother, cheb_degree
        self.gamma_D = 20.0 * p * p if gamma_D is None else gamma_D
        self.gammas = [0.1] * p if gammas is None else list(gammas)
        self.q = p + 2 if q is None else q
        self.levels = []
        for l in range(n_levels):
            Nl = N >> (n_levels - 1 - l)
            self.levels.append(LevelData(ls, d, Nl, p, self.gamma_D, self.gammas, self.q))
        self.P = [None] + [prolongation(self.levels[l].lev, self.levels[l - 1].lev)
                           for l in range(1, n_levels)]
        for l in range(1, n_levels):
            self.levels[l].patches = Patches(self.levels[l].lev, self.levels[l].A)
        A0 = self.levels[0].A.toarray()
        self.coarse_chol = sla.cho_factor(A0)
        if smoother == "chebyshev":
            for l in range(1, n_levels):
                L = self.levels[l]
                L.dinv = 1.0 / L.A.diagonal()
                L.lam_max = self.power_lambda_max(L)

    def power_lambda_max(self, L):
        """lambda_max of D^{-1} A by power iteration from the normalised
        all-ones vector: v <- w / ||w|| with w = D^{-1} A v; returns the last
        ||w|| (a fixed number of steps, so that every implementation gets the
        same estimate up to rounding)."""
        v = np.ones(L.A.shape[0])
        v /= np.linalg.norm(v)
        lam = 0.0
        for _ in range(self.CHEB_POWER_STEPS):
            w = L.dinv * (L.A @ v)
            lam = np.linalg.norm(w)
            v = w / lam
        return lam

    def chebyshev(self, l, x, b):
        """Degree-k Chebyshev smoothing of A_l x = b with point-Jacobi scaling
        on [lambda / range, lambda], lambda = safety * lambda_max(D^{-1} A)
        (three-term recurrence): k operator applications."""
        L = self.levels[l]
        lmax = self.CHEB_SAFETY * L.lam_max
        lmin = lmax / self.CHEB_RANGE
        theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
        sigma = theta / delta
        rho = 1.0 / sigma
        r = b - L.A @ x
        xp = x
        x = x + (1.0 / theta) * (L.dinv * r)
        for _ in range(1, self.cheb_degree):
            r = b - L.A @ x
            rho_new = 1.0 / (2.0 * sigma - rho)
            x, xp = x + rho_new * rho * (x - xp) + (2.0 * rho_new / delta) * (L.dinv * r), x
            rho = rho_new
        return x

    @property
    def fine(self):
        return self.levels[-1]

    def rhs(self):
        return assemble_rhs(self.fine.lev, self.gamma_D, self.q)

    def schedule(self):
        """Pre-smoothing sequence of (cut?, colour) steps (eq. "smoother-split")."""
        ncol = 1 << self.d
        seq = [(False, c) for c in range(ncol)]
        for _ in range(self.n_c):
            seq += [(True, c) for c in range(ncol)]
        return seq

    def colour_step(self, l, x, b, cut, colour):
        L = self.levels[l]
        idx = L.patches.select(cut, colour)
        if idx.size == 0:
            return x
        r = b - L.A @ x
        x = x.copy()
        P = L.patches
        for m in np.unique(P.size[idx]):
            grp = idx[P.size[idx] == m]
            Aj = np.stack([P.Aj[j] for j in grp])
            rj = np.stack([r[P.I[j]] for j in grp])
            dj = np.linalg.solve(Aj, rj[..., None])[..., 0]
            for t, j in enumerate(grp):
                x[P.I[j]] += dj[t]
        return x

    def smooth(self, l, x, b, post=False):
        if self.smoother == "chebyshev":
            return self.chebyshev(l, x, b)
        seq = self.schedule()
        if post:
            seq = seq[::-1]
        for cut, colour in seq:
            x = self.colour_step(l, x, b, cut, colour)
        return x

    def vcycle(self, b, l=None):
        """One V-cycle with zero initial guess: returns z = B_l b."""
        if l is None:
            l = len(self.levels) - 1
        if l == 0:
            return sla.cho_solve(self.coarse_chol, b)
        L = self.levels[l]
        x = np.zeros_like(b)
        x = self.smooth(l, x, b)
        r = b - L.A @ x
        xc = self.vcycle(self.P[l].T @ r, l - 1)
        x = x + self.P[l] @ xc
        x = self.smooth(l, x, b, post=True)
        return x

    def vcycle_solve(self, b, rtol=1e-9, maxit=500):
        """The V-cycle as a solver (Sec. 2.2, the direct V-cycle iteration):
        x_{k+1} = x_k + B (b - A x_k), x_0 = 0, until ||b - A x_k||_2 <=
        rtol ||b||_2.  Returns (x, iterations, history of ||r||_2)."""
        A = self.fine.A
        x = np.zeros_like(b)
        r = b.copy()
        bn = np.linalg.norm(b)
        hist = [np.linalg.norm(r)]
        it = 0
        while hist[-1] > rtol * bn and it < maxit:
            x = x + self.vcycle(r)
            r = b - A @ x
            it += 1
            hist.append(np.linalg.norm(r))
        return x, it, hist

    def gmres(self, b, rtol=1e-9, restart=30, maxit=500):
        """GMRES(restart) with the V-cycle as right preconditioner (Sec. 2.2):
        minimises ||b - A x||_2 over x_0 + B K_k(A B, r_0), x_0 = 0, Arnoldi
        by modified Gram-Schmidt, least squares by Givens rotations; stops
        when the residual norm falls to rtol ||b||_2.  Returns (x, total
        iterations, history of the residual norms)."""
        A = self.fine.A
        n = b.size
        x = np.zeros_like(b)
        bn = np.linalg.norm(b)
        r = b.copy()
        beta = np.linalg.norm(r)
        hist = [beta]
        total = 0
        while beta > rtol * bn and total < maxit:
            m = restart
            V = np.zeros((m + 1, n))
            Z = np.zeros((m, n))
            H = np.zeros((m + 1, m))
            cs, sn = np.zeros(m), np.zeros(m)
            g = np.zeros(m + 1)
            g[0] = beta
            V[0] = r / beta
            k = 0
            for j in range(m):
                Z[j] = self.vcycle(V[j])
                w = A @ Z[j]
                for i in range(j + 1):
                    H[i, j] = w @ V[i]
                    w = w - H[i, j] * V[i]
                H[j + 1, j] = np.linalg.norm(w)
                if H[j + 1, j] > 0:
                    V[j + 1] = w / H[j + 1, j]
                for i in range(j):  # earlier rotations on the new column
                    t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                    H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                    H[i, j] = t
                den = np.hypot(H[j, j], H[j + 1, j])
                cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
                H[j, j] = den
                H[j + 1, j] = 0.0
                g[j + 1] = -sn[j] * g[j]
                g[j] = cs[j] * g[j]
                k = j + 1
                total += 1
                hist.append(abs(g[j + 1]))
                if abs(g[j + 1]) <= rtol * bn or total >= maxit:
                    break
            y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
            x = x + Z[:k].T @ y
            r = b - A @ x
            beta = np.linalg.norm(r)
        return x, total, hist

    def pcg(self, b, rtol=1e-8, maxit=500):
        """CG on A_L x = b preconditioned by one V-cycle; x_0 = 0.
        Returns (x, iterations, history of ||r||_2)."""
        A = self.fine.A
        x = np.zeros_like(b)
        r = b.copy()
        bn = np.linalg.norm(b)
        hist = [np.linalg.norm(r)]
        if hist[0] <= rtol * bn:
            return x, 0, hist
        z = self.vcycle(r)
        pdir = z.copy()
        rz = r @ z
        it = 0
        while it < maxit:
            q = A @ pdir
            alpha = rz / (pdir @ q)
            x = x + alpha * pdir
            r = r - alpha * q
            it += 1
            hist.append(np.linalg.norm(r))
            if hist[-1] <= rtol * bn:
                break
            z = self.vcycle(r)
            rz_new = r @ z
            beta = rz_new / rz
            rz = rz_new
            pdir = z + beta * pdir
        return x, it, hist
