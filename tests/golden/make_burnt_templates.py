"""Writes burnt_templates_mech100.npz: equilibrium states of the 100-species / 700-reaction
synthetic mechanism (seed 3) for the burnt cells of the uneven-stiffness workload.

Each template draws T ~ U[2000, 2400] K and the element totals of a Dirichlet(1) composition,
then takes the ideal-gas Gibbs minimum at (T, 60 atm) by the element-potential method
(n_k = N exp(-g_k/RT - ln(p/Patm) + sum_e lambda_e a_ek), sum_k n_k = N, element balance), with
g_k/RT from the oracle's NASA-7 thermo.  Run:  python tests/golden/make_burnt_templates.py
"""
import os
import sys

import numpy as np
from scipy.optimize import fsolve

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2105_12070_gb300 import synth  # noqa: E402  (input generator only)

P_ATM = 60.0


def gibbs_equilibrium(ora, comp, W, T, b):
    _, hRT, sR = ora.thermo(T)
    g = hRT - sR
    A = comp.T.astype(float)
    E = A.shape[0]
    lnp = np.log(P_ATM)

    def resid(x):
        lam, lnN = x[:E], x[E]
        lnx = np.clip(-g - lnp + lam @ A, -700, 700)
        xk = np.exp(lnx)
        return np.concatenate([(A @ (np.exp(lnN) * xk) - b) / b, [xk.sum() - 1.0]])

    rng = np.random.default_rng(int(T * 1000) % 2 ** 31)
    for trial in range(200):
        x0 = np.concatenate([rng.normal(0.0, 20.0, E), [np.log(b.sum()) + rng.normal(0, 1)]])
        x, info, ier, _ = fsolve(resid, x0, full_output=True, xtol=1e-14, maxfev=20000)
        if ier == 1 and np.abs(resid(x)).max() < 1e-10:
            lnx = -g - lnp + x[:E] @ A
            xk = np.exp(lnx)
            y = xk * W
            return y / y.sum()
    return None


def main(n_templates=32):
    mech = synth.mechanism_100()
    ora = oracle.OracleMechanism(mech.write_temp())
    rng = np.random.default_rng(303)
    Ts, Ys = [], []
    while len(Ts) < n_templates:
        T = rng.uniform(2000.0, 2400.0)
        y0 = rng.dirichlet(np.ones(mech.K))
        b = mech.comp.T @ (y0 / mech.W)
        y = gibbs_equilibrium(ora, mech.comp, mech.W, T, b)
        if y is None:
            continue
        Ts.append(T)
        Ys.append(y)
        print(len(Ts), T, np.sort(y)[-3:], flush=True)
    np.savez_compressed(os.path.join(HERE, "burnt_templates_mech100.npz"), T=np.array(Ts), Y=np.array(Ys),
                        p_atm=P_ATM)


if __name__ == "__main__":
    main()
