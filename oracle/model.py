"""Floating-base (centroidal) model of one agent and its linearisation.

Paper: Sec. III-A, Eq. (base_dynamics) and its footnote (projected to the
centre of mass it is the centroidal dynamics); the decision variables of
Eq. (mpc_formulation) are positions, velocities and contact forces.  The
reading used here keeps the joint velocities as inputs:

  state x = [p(3), Theta(3) = (roll, pitch, yaw), v(3) world, w(3) world, q(18)]
  input u = [f_L(3), m_L(3), f_R(3), m_R(3), qdot(18)]      (world frame)

  p_dot     = v
  Theta_dot = E(Theta)^-1 w         (ZYX Euler-rate map)
  v_dot     = (f_L + f_R)/m + g,    g = (0, 0, -9.81)
  w_dot     = I_w^-1 (sum_i r_i(q) x f_i + m_i - w x I_w w)
  q_dot     = qdot
  r_i(q)    = lever_i + J_leg_i[0:3] (q_leg_i - q_nom_leg_i)

I_w = R(Theta0) diag(I_b) R(Theta0)^T is frozen at the linearisation point.
Discretisation is forward Euler, linearised about (x0, u_ref_k) (real-time
iteration, Sec. II-A / III-B): x_{k+1} = A_k x_k + B_k u_k + c_k with
A_k = I + dt f_x, B_k = dt f_u, c_k = dt (f - f_x x0 - f_u u_ref_k).
Jacobians are taken by complex step (Squire & Trapp 1998).

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import numpy as np

GRAVITY = 9.81


def rot_x(a):
    c, s = np.cos(a), np.sin(a)
    one, zero = np.ones_like(c), np.zeros_like(c)
    return np.array([[one, zero, zero], [zero, c, -s], [zero, s, c]])


def rot_y(a):
    c, s = np.cos(a), np.sin(a)
    one, zero = np.ones_like(c), np.zeros_like(c)
    return np.array([[c, zero, s], [zero, one, zero], [-s, zero, c]])


def rot_z(a):
    c, s = np.cos(a), np.sin(a)
    one, zero = np.ones_like(c), np.zeros_like(c)
    return np.array([[c, -s, zero], [s, c, zero], [zero, zero, one]])


def rotation(theta):
    """R = Rz(yaw) Ry(pitch) Rx(roll): body -> world."""
    return rot_z(theta[2]) @ rot_y(theta[1]) @ rot_x(theta[0])


def euler_rate_matrix(theta):
    """E(Theta) with w_world = E(Theta) Theta_dot, built from its definition.

    w = yaw_dot e_z + pitch_dot Rz(yaw) e_y + roll_dot Rz(yaw) Ry(pitch) e_x,
    so the columns of E are those three axes.
    """
    ex = np.array([1.0, 0.0, 0.0])
    ey = np.array([0.0, 1.0, 0.0])
    ez = np.array([0.0, 0.0, 1.0])
    col_roll = rot_z(theta[2]) @ rot_y(theta[1]) @ ex
    col_pitch = rot_z(theta[2]) @ ey
    col_yaw = ez + 0.0 * theta[2]
    return np.stack([col_roll, col_pitch, col_yaw], axis=1)


def cross(a, b):
    return np.array([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


def world_inertia(model, theta0):
    """I_w = R(Theta0) diag(I_b) R(Theta0)^T (real, frozen)."""
    R = rotation(np.asarray(theta0, dtype=float))
    return R @ np.diag(model["inertia"]) @ R.T


def foot_lever(model, q, foot):
    """r_i(q) = lever_i + J_leg_i[0:3] (q_leg_i - q_nom_leg_i)."""
    sl = slice(5 * foot, 5 * foot + 5)
    return model["lever"][foot] + model["J_leg"][foot][0:3] @ (q[sl] - model["q_nom"][sl])


def dynamics(model, x, u, Iw):
    """Continuous-time f(x, u); complex-step safe (no abs, no branches)."""
    v = x[6:9]
    w = x[9:12]
    q = x[12:30]
    dtype = np.result_type(x, u)
    f = np.zeros(30, dtype=dtype)
    f[0:3] = v
    f[3:6] = np.linalg.solve(euler_rate_matrix(x[3:6]), w)
    fL, mL, fR, mR = u[0:3], u[3:6], u[6:9], u[9:12]
    f[6:9] = (fL + fR) / model["mass"] + np.array([0.0, 0.0, -GRAVITY])
    rL = foot_lever(model, q, 0)
    rR = foot_lever(model, q, 1)
    torque = cross(rL, fL) + mL + cross(rR, fR) + mR - cross(w, Iw @ w)
    f[9:12] = np.linalg.solve(Iw, torque)
    f[12:30] = u[12:30]
    return f


def jacobians(model, x_bar, u_bar, Iw, h=1e-30):
    """(f, f_x, f_u) at (x_bar, u_bar) by complex step."""
    x_bar = np.asarray(x_bar, dtype=float)
    u_bar = np.asarray(u_bar, dtype=float)
    f0 = dynamics(model, x_bar, u_bar, Iw).real
    fx = np.empty((30, 30))
    fu = np.empty((30, 30))
    for j in range(30):
        xc = x_bar.astype(complex)
        xc[j] += 1j * h
        fx[:, j] = dynamics(model, xc, u_bar.astype(complex), Iw).imag / h
        uc = u_bar.astype(complex)
        uc[j] += 1j * h
        fu[:, j] = dynamics(model, x_bar.astype(complex), uc, Iw).imag / h
    return f0, fx, fu


def linearise(model, x0, u_ref):
    """Discrete affine model for every stage: lists A[k], B[k], c[k].

    u_ref: (N, 30) input references, the linearisation inputs of each stage.
    """
    dt = float(model["dt"])
    Iw = world_inertia(model, x0[3:6])
    A, B, c = [], [], []
    for k in range(u_ref.shape[0]):
        f0, fx, fu = jacobians(model, x0, u_ref[k], Iw)
        A.append(np.eye(30) + dt * fx)
        B.append(dt * fu)
        c.append(dt * (f0 - fx @ x0 - fu @ u_ref[k]))
    return A, B, c
