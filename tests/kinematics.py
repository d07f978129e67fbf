"""Test-only relativistic kinematics for planted-truth events (FP64 numpy).

Independent of both the oracle and the CUDA path: two-body decays in the
parent rest frame followed by a Lorentz boost, so that the true masses and
neutrino momenta of a constructed event are known by construction.
"""
import numpy as np


def p4(px, py, pz, m):
    return np.array([px, py, pz, np.sqrt(px * px + py * py + pz * pz + m * m)])


def boost(v, beta):
    """Boost four-vector v = (px, py, pz, E) by velocity beta (3-vector)."""
    beta = np.asarray(beta, dtype=np.float64)
    b2 = float(beta @ beta)
    if b2 == 0.0:
        return v.copy()
    g = 1.0 / np.sqrt(1.0 - b2)
    p = v[:3]
    bp = float(beta @ p)
    g2 = (g - 1.0) / b2
    p_new = p + g2 * bp * beta + g * beta * v[3]
    e_new = g * (v[3] + bp)
    return np.array([p_new[0], p_new[1], p_new[2], e_new])


def two_body(parent, m1, m2, rng):
    """Decay `parent` (four-vector) into daughters of masses m1, m2 with an
    isotropic direction in the parent rest frame."""
    M2 = parent[3] ** 2 - parent[:3] @ parent[:3]
    M = np.sqrt(M2)
    pstar = np.sqrt((M2 - (m1 + m2) ** 2) * (M2 - (m1 - m2) ** 2)) / (2.0 * M)
    cth = rng.uniform(-1, 1)
    sth = np.sqrt(1 - cth * cth)
    ph = rng.uniform(-np.pi, np.pi)
    n = np.array([sth * np.cos(ph), sth * np.sin(ph), cth])
    d1 = np.concatenate([pstar * n, [np.sqrt(pstar ** 2 + m1 * m1)]])
    d2 = np.concatenate([-pstar * n, [np.sqrt(pstar ** 2 + m2 * m2)]])
    beta = parent[:3] / parent[3]
    return boost(d1, beta), boost(d2, beta)


def minkowski_m2(v):
    return v[3] ** 2 - v[:3] @ v[:3]


def random_parent(M, rng, pmax=300.0):
    p = rng.uniform(-pmax, pmax, 3)
    return p4(p[0], p[1], p[2], M)
