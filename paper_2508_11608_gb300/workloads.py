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
    "disk2d_q1_n64": dict(dim=2, n_cells=64, n_levels=4, degree=1, center=[0.031, 0.017], radius=0.7),
}


def random_vector(n, seed):
    """Seeded standard-normal FP64 vector."""
    return np.random.default_rng(seed).standard_normal(n)


def problem_kwargs(name):
    c = CONFIGS[name]
    return dict(dim=c["dim"], n_cells=c["n_cells"], n_levels=c["n_levels"], degree=c["degree"],
                center=c["center"], radius=c["radius"])
