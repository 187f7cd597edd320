"""Semi-analytic Runge-Kutta (SARK) coefficients (oracle; test infrastructure only).

Paper, Sec. 4: with dq/dt = -Lambda q + F(q) and gamma = -dt/tau, the stages are
    q_i     = exp(c_i gamma) q_n + dt sum_{j<i} atilde_ij F_j,
    q_{n+1} = exp(gamma)     q_n + dt sum_j   btilde_j  F_j,
with c = (0, 1/2, 1/2, 1) from the classical RK4 tableau (Table 1) and the
atilde, btilde printed in closed form in Sec. 4.  This module evaluates those
printed closed forms exactly as printed, in 60-digit arithmetic (mpmath), and
rounds the results to FP64, so the catastrophic cancellation of the printed
forms at small |gamma| does not reach the oracle.  At gamma = 0 (fields 1..3,
Lambda = 0) the scheme is the base RK4 method (the non-stiff limit stated in
Sec. 4).

Reading (garbled constraint): the printed stage-sum constraint carries a
spurious 1/c_i; the printed coefficients satisfy
sum_j atilde_ij = gamma^-1 (exp(c_i gamma) - 1), which is what the GCL argument
of Sec. 5 needs, and that is the form the tests check.

Pins: gamma -> 0 gives RK4; sum identities; the scalar problem
y' = -y/tau + g (g constant) is integrated exactly; fourth-order convergence on
y' = -y/tau + sin t.
"""
import mpmath as mp

RK4_C = (0.0, 0.5, 0.5, 1.0)
RK4_A = ((0.0, 0.0, 0.0, 0.0),
         (0.5, 0.0, 0.0, 0.0),
         (0.0, 0.5, 0.0, 0.0),
         (0.0, 0.0, 1.0, 0.0))
RK4_B = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


def sark_coefficients(gamma):
    """Return (E, A, B): stage exponentials E[i] = exp(c_i gamma) for i = 0..3 and
    E[4] = exp(gamma) (final), the 4x4 strictly lower atilde, and btilde.

    gamma = 0 returns the RK4 tableau with unit exponentials.
    """
    if gamma == 0.0:
        return ([1.0] * 5, [list(row) for row in RK4_A], list(RK4_B))
    with mp.workdps(60):
        g = mp.mpf(gamma)
        eh = mp.exp(g / 2)
        e1 = mp.exp(g)
        a10 = (-1 + eh) / g
        a20 = (4 + g + eh * (g - 4)) / g ** 2
        a21 = (-4 - 2 * g + 4 * eh) / g ** 2
        a30 = (2 + g + e1 * (g - 2)) / g ** 2
        a31 = mp.mpf(0)
        a32 = (-2 - 2 * g + 2 * e1) / g ** 2
        b0 = (-4 - g + e1 * (g ** 2 - 3 * g + 4)) / g ** 3
        b1 = (4 + 2 * g + e1 * (2 * g - 4)) / g ** 3
        b2 = (4 + 2 * g + e1 * (2 * g - 4)) / g ** 3
        b3 = (-4 - 3 * g - g ** 2 + e1 * (4 - g)) / g ** 3
        E = [1.0, float(eh), float(eh), float(e1), float(e1)]
        A = [[0.0, 0.0, 0.0, 0.0],
             [float(a10), 0.0, 0.0, 0.0],
             [float(a20), float(a21), 0.0, 0.0],
             [float(a30), float(a31), float(a32), 0.0]]
        B = [float(b0), float(b1), float(b2), float(b3)]
    return E, A, B


def sark_scalar_step(y, t, dt, tau, f):
    """One SARK step of y' = -y/tau + f(y, t) (tau = inf allowed): the scheme of
    Sec. 4 applied to a scalar; used by the tests only."""
    gamma = 0.0 if tau == float('inf') else -dt / tau
    E, A, B = sark_coefficients(gamma)
    F = []
    for i in range(4):
        yi = E[i] * y + dt * sum(A[i][j] * F[j] for j in range(i))
        F.append(f(yi, t + RK4_C[i] * dt))
    return E[4] * y + dt * sum(B[j] * F[j] for j in range(4))
