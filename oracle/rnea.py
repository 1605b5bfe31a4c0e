"""Inverse dynamics of a floating-base kinematic tree by the spatial recursive
Newton-Euler algorithm (paper Sec. III-C, Eq. (rnea): tau_RNEA = M(q) qddot +
h(q, qdot) - J^T F, the first two terms computed by RNEA; Featherstone,
"Rigid Body Dynamics Algorithms", 2008, Ch. 2 spatial algebra and Ch. 5
Table 5.1 recursive Newton-Euler).

Spatial vectors in Plucker coordinates, body frames: motion m = [w; v] (v the
velocity of the body point at the frame origin), force f = [n; f].  Joint i is
revolute about a unit axis a_i given in its parent link's frame, located at
offset p_i from the parent frame's origin; link i's frame is the parent's
translated to the joint and rotated by q_i about a_i.  The base's motion is
prescribed (floating base, known acceleration): its spatial velocity and
acceleration enter the recursion at the root, and gravity is added as an
upward acceleration of the root (Featherstone Sec. 5.3).

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .model import GRAVITY


def skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def rot_axis(a, q):
    """Active rotation by angle q about unit axis a (Rodrigues)."""
    a = np.asarray(a, float)
    K = skew(a)
    return np.eye(3) + np.sin(q) * K + (1.0 - np.cos(q)) * (K @ K)


def xrot(E):
    """Plucker transform of a pure change of orientation (E: A -> B coordinates)."""
    X = np.zeros((6, 6))
    X[:3, :3] = E
    X[3:, 3:] = E
    return X


def xlt(p):
    """Plucker transform to a frame whose origin sits at p (same orientation)."""
    X = np.eye(6)
    X[3:, :3] = -skew(p)
    return X


def crm(v):
    """Motion cross product operator v x_m."""
    X = np.zeros((6, 6))
    X[:3, :3] = skew(v[:3])
    X[3:, :3] = skew(v[3:])
    X[3:, 3:] = skew(v[:3])
    return X


def crf(v):
    """Force cross product operator v x_f = -(v x_m)^T."""
    return -crm(v).T


def spatial_inertia(m, c, Ic):
    """Spatial inertia at the frame origin of a body of mass m, centre of mass
    c and rotational inertia Ic about the centre of mass (Featherstone Eq. 2.63)."""
    C = skew(c)
    I = np.zeros((6, 6))
    I[:3, :3] = Ic + m * C @ C.T
    I[:3, 3:] = m * C
    I[3:, :3] = m * C.T
    I[3:, 3:] = m * np.eye(3)
    return I


def rnea(parent, axis, offset, mass, com, inertia, q, qd, qdd, *, base_R=None, base_w=None, base_v=None,
         base_dw=None, base_a=None, gravity=GRAVITY):
    """Joint torques of a tree (parents listed before children; parent -1 =
    the base).  inertia: per link the diagonal of its rotational inertia about
    its centre of mass, or a full 3x3.  Base quantities in world coordinates:
    orientation base_R (body -> world), angular velocity base_w, velocity of
    the base origin base_v, angular acceleration base_dw and classical
    acceleration of the base origin base_a (all zero by default: a fixed base).
    Gravity acts along -z of the world."""
    n = len(parent)
    R = np.eye(3) if base_R is None else np.asarray(base_R, float)
    z3 = np.zeros(3)
    w = z3 if base_w is None else np.asarray(base_w, float)
    vb = z3 if base_v is None else np.asarray(base_v, float)
    dw = z3 if base_dw is None else np.asarray(base_dw, float)
    ab = z3 if base_a is None else np.asarray(base_a, float)
    Rt = R.T
    v0 = np.concatenate([Rt @ w, Rt @ vb])
    # spatial acceleration of the base (linear part: a_O - w x v_O), minus gravity
    a0 = np.concatenate([Rt @ dw, Rt @ (ab - np.cross(w, vb) + np.array([0.0, 0.0, gravity]))])
    X, S, v, a, f = [None] * n, [None] * n, [None] * n, [None] * n, [None] * n
    for i in range(n):
        ax = np.asarray(axis[i], float)
        X[i] = xrot(rot_axis(ax, q[i]).T) @ xlt(offset[i])
        S[i] = np.concatenate([ax, z3])
        vp = v0 if parent[i] < 0 else v[parent[i]]
        ap = a0 if parent[i] < 0 else a[parent[i]]
        v[i] = X[i] @ vp + S[i] * qd[i]
        a[i] = X[i] @ ap + S[i] * qdd[i] + crm(v[i]) @ S[i] * qd[i]
        Ic = np.asarray(inertia[i], float)
        Ic = np.diag(Ic) if Ic.ndim == 1 else Ic
        I = spatial_inertia(float(mass[i]), np.asarray(com[i], float), Ic)
        f[i] = I @ a[i] + crf(v[i]) @ I @ v[i]
    tau = np.zeros(n)
    for i in range(n - 1, -1, -1):
        tau[i] = S[i] @ f[i]
        if parent[i] >= 0:
            f[parent[i]] = f[parent[i]] + X[i].T @ f[i]
    return tau


def chain_parents(chains, n):
    """Parent list of a tree made of chains hanging off the base: (first
    joint, length) per chain."""
    parent = [-1] * n
    for j0, length in chains:
        for t in range(1, length):
            parent[j0 + t] = j0 + t - 1
    return parent
