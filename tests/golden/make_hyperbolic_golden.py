"""Writes hyperbolic_closed_forms.txt: closed-form footpoint Q, perpendicular Q,
length and exit face for seeds on z = 0 in the linear hyperbolic field
B = (lam x, -lam y, B0), lam = 3, B0 = 1, box [-1,1]^2 x [0,1].

Pure mathematics (numpy/scipy): it calls neither the oracle nor the CUDA path.
Derivation: the flow map of dx/dt = B is (x0 e^{lam t}, y0 e^{-lam t}, B0 t);
lines with |x0| < e^{-lam/B0} leave through z = 1 at t = 1/B0, others through
x = +-1 at t = ln(1/|x0|)/lam. Footpoint Q (Jacobian of the boundary map):
k^2 + k^-2 (k = e^{lam/B0}) for top exits, lam (x0^2 + y0^2)/B0 + B0/(lam x0^2)
for side exits. Perpendicular Q (Eq. finalQ with dx_perp):
||P_e D [a b]||_F^2 |B_e| / |B_s|, D = diag(e^{lam t}, e^{-lam t}, 1).
Length: integral of |B(x(t))| dt.
"""
import math
import os

import numpy as np
from scipy import integrate

LAM, B0 = 3.0, 1.0


def closed_forms(x0, y0):
    k = math.exp(LAM / B0)
    if abs(x0) < math.exp(-LAM / B0):
        te, qf, face = 1.0 / B0, k * k + 1.0 / (k * k), 5
    else:
        te = math.log(1.0 / abs(x0)) / LAM
        qf = LAM * (x0 * x0 + y0 * y0) / B0 + B0 / (LAM * x0 * x0)
        face = 1 if x0 > 0 else 0
    Bs = np.array([LAM * x0, -LAM * y0, B0])
    D = np.diag([math.exp(LAM * te), math.exp(-LAM * te), 1.0])
    Be = D @ Bs
    u = Bs / np.linalg.norm(Bs)
    t = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    a = np.cross(u, t)
    a /= np.linalg.norm(a)
    b = np.cross(u, a)
    ue = Be / np.linalg.norm(Be)
    M = (np.eye(3) - np.outer(ue, ue)) @ D @ np.column_stack([a, b])
    qp = float(np.sum(M * M)) * np.linalg.norm(Be) / np.linalg.norm(Bs)
    L, _ = integrate.quad(lambda s: math.sqrt((LAM * x0) ** 2 * math.exp(2 * LAM * s)
                                              + (LAM * y0) ** 2 * math.exp(-2 * LAM * s) + B0 ** 2),
                          0.0, te, epsabs=1e-14, epsrel=1e-13, limit=200)
    return qf, qp, L, face


def main():
    # pixel centres of the 256 x 256 map on z = 0 (u = (2,0,0), v = (0,2,0))
    rows = []
    for j in range(0, 256, 17):
        for i in list(range(0, 256, 23)) + list(range(122, 134, 3)):
            x0 = -1 + (i + 0.5) * 2 / 256
            y0 = -1 + (j + 0.5) * 2 / 256
            qf, qp, L, face = closed_forms(x0, y0)
            rows.append((i, j, x0, y0, qf, qp, L, face))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hyperbolic_closed_forms.txt")
    with open(path, "w") as f:
        f.write("# Closed forms for the linear hyperbolic field (lam=3, B0=1), seeds on z=0;\n")
        f.write("# written by tests/golden/make_hyperbolic_golden.py (mathematics only).\n")
        f.write("# Q definitions: Eq. finalQ (perpendicular) and its footpoint variant.\n")
        f.write("# i j x0 y0 Q_foot Q_perp L exit_face\n")
        for r in rows:
            f.write("%d %d %.17g %.17g %.17g %.17g %.17g %d\n" % r)


if __name__ == "__main__":
    main()
