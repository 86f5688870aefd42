"""Synthetic workloads and seeded input generators.

Holds none of the method's arithmetic: only problem definitions (geometry,
mesh, degree, levels) and seeded random vectors, shared by the tests, the
smoke check and the benchmark."""

import numpy as np

# Level-set domains cut out of [-1, 1]^d (the method's model problem, Sec. 2,
# with the manufactured solution u = prod sin(pi x_k)).
CONFIGS = {
    # 2D disk r = 0.7 at (0.031, 0.017), 32^2 cells, Q2, 3 levels
    "disk2d_q2_n32": dict(dim=2, n_cells=32, n_levels=3, degree=2, center=[0.031, 0.017], radius=0.7),
    # 3D ball r = 0.7 at (0.05, 0.03, 0.02), 64^3 cells, Q2, 5 levels
    "ball3d_q2_n64": dict(dim=3, n_cells=64, n_levels=5, degree=2, center=[0.05, 0.03, 0.02], radius=0.7),
    # the same ball at 128^3 cells, 6 levels
    "ball3d_q2_n128": dict(dim=3, n_cells=128, n_levels=6, degree=2, center=[0.05, 0.03, 0.02], radius=0.7),
    # the same ball at 224^3 cells, 6 levels (about 17M active DoFs)
    "ball3d_q2_n224": dict(dim=3, n_cells=224, n_levels=6, degree=2, center=[0.05, 0.03, 0.02], radius=0.7),
    # small cases spanning several patches, tiles and ragged tails
    "ball3d_q2_n16": dict(dim=3, n_cells=16, n_levels=3, degree=2, center=[0.05, 0.03, 0.02], radius=0.7),
    "ball3d_q2_n32": dict(dim=3, n_cells=32, n_levels=4, degree=2, center=[0.05, 0.03, 0.02], radius=0.7),
    "ball3d_q1_n16": dict(dim=3, n_cells=16, n_levels=3, degree=1, center=[0.05, 0.03, 0.02], radius=0.7),
    "disk2d_q3_n32": dict(dim=2, n_cells=32, n_levels=3, degree=3, center=[0.031, 0.017], radius=0.7),
    # degree 4 (beyond the paper's Q3)
    "disk2d_q4_n32": dict(dim=2, n_cells=32, n_levels=3, degree=4, center=[0.031, 0.017], radius=0.7),
    "disk2d_q1_n64": dict(dim=2, n_cells=64, n_levels=4, degree=1, center=[0.031, 0.017], radius=0.7),
}


def random_vector(n, seed):
    """Seeded standard-normal FP64 vector."""
    return np.random.default_rng(seed).standard_normal(n)


def problem_kwargs(name):
    c = CONFIGS[name]
    return dict(dim=c["dim"], n_cells=c["n_cells"], n_levels=c["n_levels"], degree=c["degree"],
                center=c["center"], radius=c["radius"])


def flower_batch(count=256, seed=20260101, sizes=(32, 64, 128, 256), degrees=(2, 3), coarsest=8):
    """Seeded batch of 2D instances: flower curves r(theta) = 0.6 + 0.1 cos(m
    (theta - theta_0)) with m in {3..7}, theta_0 uniform, centre offset uniform
    in the disk of radius 0.05; N uniform over `sizes`, degree uniform over
    `degrees`, levels so that the coarsest mesh has `coarsest` cells per
    direction.  Returns a list of Problem keyword dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.integers(3, 8))
        t0 = float(rng.uniform(0.0, 2.0 * np.pi))
        rad = 0.05 * np.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * np.pi)
        c = [float(rad * np.cos(ang)), float(rad * np.sin(ang))]
        N = int(rng.choice(sizes))
        p = int(rng.choice(degrees))
        L = int(np.log2(N // coarsest)) + 1
        out.append(dict(dim=2, n_cells=N, n_levels=L, degree=p,
                        levelset={"kind": "flower", "center": c, "lobes": m, "phase": t0}))
    return out


def rotation(a, b, c):
    """Rotation matrix R_z(a) R_y(b) R_x(c) as nested lists."""
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rx = np.array([[1, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return (Rz @ Ry @ Rx).tolist()


def serving_requests(count=500, seed=20260102, sizes=(32, 48, 64, 96)):
    """Seeded stream of 3D solve requests: spheres (r in [0.4, 0.8], centre
    offset <= 0.05), ellipsoids (semi-axes in [0.4, 0.8], random rotation)
    and tori (R = 0.6, r = 0.2, random axis); Q2; N uniform over `sizes`;
    levels so that the coarsest mesh has 4..8 cells per direction (tori at
    least 8).  Returns Problem keyword dicts (arrival times are drawn by the
    server from its own seeded generator)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        kind = ["sphere", "ellipsoid", "torus"][int(rng.integers(0, 3))]
        N = int(rng.choice(sizes))
        off = rng.uniform(-1, 1, 3)
        off = (0.05 * rng.uniform() ** (1 / 3) * off / max(np.linalg.norm(off), 1e-12)).tolist()
        if kind == "sphere":
            ls = {"kind": "sphere", "center": off, "radius": float(rng.uniform(0.4, 0.8))}
        elif kind == "ellipsoid":
            ls = {"kind": "ellipsoid", "center": off, "axes": rng.uniform(0.4, 0.8, 3).tolist(),
                  "rot": rotation(*rng.uniform(0, 2 * np.pi, 3))}
        else:
            ls = {"kind": "torus", "center": off, "rot": rotation(*rng.uniform(0, 2 * np.pi, 3)),
                  "major": 0.6, "minor": 0.2}
        n0_min = 8 if kind == "torus" else 4
        L = 1
        while N % (2 ** L) == 0 and N // (2 ** L) >= n0_min:
            L += 1
        out.append(dict(dim=3, n_cells=N, n_levels=L, degree=2, levelset=ls))
    return out
