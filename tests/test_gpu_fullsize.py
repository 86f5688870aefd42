"""Parity at the benchmark's full size (3D Q2 ball, 64^3 cells, 5 levels,
435,603 DoFs), in the launch configuration bench.py times.

The oracle cannot assemble and solve this size in test time, so it computes
sampled outputs one by one: the row (A x)_i of a DoF from the oracle's own
element matrices (uncut stiffness, cut-cell volume + Nitsche terms by the
cut-cell rule) and ghost-face matrices of the cells and faces around that DoF
(Sec. 2.1).  Properties that hold at any size cover the rest: A and the
V-cycle B are symmetric, and the solves reach the 1e-8 residual with the
residual entries of the final iterate confirmed by oracle rows."""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2508_11608_gb300 as cm  # noqa: E402
from paper_2508_11608_gb300.workloads import CONFIGS, problem_kwargs, random_vector  # noqa: E402
from oracle.fem import Level, cut_cell_matrix, ghost_face_matrix, uncut_stiffness  # noqa: E402
from oracle.levelset import Sphere  # noqa: E402

DEV = "cuda:0"
NAME = "ball3d_q2_n64"
GAMMA_D, GAMMAS, QUAD = 80.0, [0.1, 0.1], 4  # 20 p^2, gamma_k = 0.1, q = p + 2


class OracleRows:
    """(A x)_i for single DoFs from the oracle's cell and face matrices."""

    def __init__(self, cfg):
        self.lev = Level(Sphere(cfg["center"], cfg["radius"]), cfg["dim"], cfg["n_cells"], cfg["degree"])
        self.Kref = uncut_stiffness(self.lev)
        self.Gref = [ghost_face_matrix(self.lev, k, GAMMAS) for k in range(self.lev.d)]
        self.faces = self.lev.ghost_faces()
        self.cut_cache = {}
        self.faces_of_cell = {}
        for f in self.faces:
            for c in f[1:]:
                self.faces_of_cell.setdefault(c, []).append(f)

    def cells_of_node(self, node):
        lev = self.lev
        idx = np.array([(node // lev.n ** k) % lev.n for k in range(lev.d)])
        opts = []
        for k in range(lev.d):
            a, r = divmod(int(idx[k]), lev.p)
            o = [a] if r else [a - 1, a]
            opts.append([c for c in o if 0 <= c < lev.N])
        out = []
        for c0 in opts[0]:
            for c1 in opts[1]:
                for c2 in opts[2]:
                    out.append(c0 + lev.N * (c1 + lev.N * c2))
        return out

    def matrix(self, c):
        if not self.lev.cut[c]:
            return self.Kref
        if c not in self.cut_cache:
            self.cut_cache[c] = cut_cell_matrix(self.lev, c, GAMMA_D, QUAD)
        return self.cut_cache[c]

    def row_times(self, dof, x):
        lev = self.lev
        node = int(lev.dof_nodes[dof])
        acc = 0.0
        scale = 0.0
        cells = [c for c in self.cells_of_node(node) if lev.active[c]]
        for c in cells:
            nodes = lev.cell_nodes[c]
            i = int(np.nonzero(nodes == node)[0][0])
            K = self.matrix(c)
            xv = x[lev.node_to_dof[nodes]]
            acc += K[i] @ xv
            scale += np.abs(K[i]) @ np.abs(xv)
        seen = set()
        for c in cells:
            for f in self.faces_of_cell.get(c, []):
                if f in seen:
                    continue
                seen.add(f)
                k, c1, c2 = f
                nodes = np.concatenate([lev.cell_nodes[c1], lev.cell_nodes[c2]])
                G = self.Gref[k]
                xv = x[lev.node_to_dof[nodes]]
                for i in np.nonzero(nodes == node)[0]:
                    acc += G[i] @ xv
                    scale += np.abs(G[i]) @ np.abs(xv)
        return acc, scale


@pytest.fixture(scope="module")
def setup():
    cfg = CONFIGS[NAME]
    pb = cm.Problem(**problem_kwargs(NAME))
    orc = OracleRows(cfg)
    assert pb.n_dofs() == orc.lev.ndof
    rng = np.random.default_rng(11)
    near_cut = np.unique(orc.lev.node_to_dof[orc.lev.cell_nodes[np.nonzero(orc.lev.cut)[0]]].ravel())
    near_cut = near_cut[near_cut >= 0]
    sample = np.concatenate([rng.choice(near_cut, 24, replace=False),
                             rng.choice(orc.lev.ndof, 8, replace=False)])
    return pb, orc, sample


def test_sampled_operator_rows_match_the_oracle(setup):
    pb, orc, sample = setup
    n = pb.n_dofs()
    xh = random_vector(n, 2024)
    x = torch.tensor(xh, device=DEV)
    y = torch.zeros_like(x)
    pb.apply(x, y)
    torch.cuda.synchronize()
    yh = y.cpu().numpy()
    for i in sample:
        ref, scale = orc.row_times(int(i), xh)
        assert abs(yh[i] - ref) <= 1e-12 * scale, (int(i), yh[i], ref)


def test_operator_and_vcycle_are_symmetric_at_full_size(setup):
    pb, _, _ = setup
    n = pb.n_dofs()
    u = torch.tensor(random_vector(n, 1), device=DEV)
    v = torch.tensor(random_vector(n, 2), device=DEV)
    Au, Av = torch.zeros_like(u), torch.zeros_like(u)
    pb.apply(u, Au)
    pb.apply(v, Av)
    a, b = torch.dot(Au, v).item(), torch.dot(u, Av).item()
    assert abs(a - b) <= 1e-12 * (Au.norm() * v.norm()).item()
    pb.set_precision(cm.CF_FP64)
    Bu, Bv = torch.zeros_like(u), torch.zeros_like(u)
    pb.vcycle(u, Bu)
    pb.vcycle(v, Bv)
    a, b = torch.dot(Bu, v).item(), torch.dot(u, Bv).item()
    assert abs(a - b) <= 1e-11 * (Bu.norm() * v.norm()).item()
    assert torch.dot(Bu, u).item() > 0.0


@pytest.mark.parametrize("prec", [cm.CF_FP64, cm.CF_MIXED])
def test_full_size_solve_residual_confirmed_by_oracle_rows(setup, prec):
    pb, orc, sample = setup
    n = pb.n_dofs()
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    pb.rhs(b)
    pb.set_precision(prec)
    info = pb.solve(b, x, rtol=1e-8)
    torch.cuda.synchronize()
    assert info["true_rel_residual"] <= 1e-8
    bh, xh = b.cpu().numpy(), x.cpu().numpy()
    bnorm = np.linalg.norm(bh)
    # sampled residual entries from the oracle rows agree with a 1e-8 residual
    for i in sample:
        ax, scale = orc.row_times(int(i), xh)
        assert abs(bh[i] - ax) <= 1e-8 * bnorm + 1e-12 * scale


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ball3d_q2_n64_pcg.npz")


@pytest.mark.parametrize("prec", [cm.CF_FP64, cm.CF_MIXED])
def test_full_size_solve_matches_the_oracle_solution(setup, prec):
    """Full-vector parity at the benchmark's size: the oracle's PCG solution
    of the same problem (stored, written by tests/golden/make_ball64_solution.py
    from oracle/ alone).  FP64: CG iterations within one and relative L2
    difference 1e-10.  Mixed: the same final residual; its distance to the
    FP64 oracle solution is that of two 1e-8-residual solutions (bounded by
    1e-6 here, the measured value is printed)."""
    pb, _, _ = setup
    g = np.load(GOLDEN)
    xo = g["x"]
    n = pb.n_dofs()
    assert n == xo.size
    b = torch.zeros(n, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    pb.rhs(b)
    pb.set_precision(prec)
    try:
        info = pb.solve(b, x, rtol=1e-8)
    finally:
        pb.set_precision(cm.CF_FP64)
    torch.cuda.synchronize()
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    print(f"precision {prec}: {info['iterations']} iterations (oracle {int(g['iterations'])}), "
          f"relative L2 difference to the oracle {err:.3e}")
    assert info["true_rel_residual"] <= 1.01e-8
    if prec == cm.CF_FP64:
        assert abs(info["iterations"] - int(g["iterations"])) <= 1
        assert err <= 1e-10
    else:
        assert info["iterations"] <= int(g["iterations"]) + 2
        assert err <= 1e-6
