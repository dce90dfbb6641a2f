"""FP64 oracle: PiTSBiCG (Algorithm 1) and the parareal baseline (eq. (6)).

TEST INFRASTRUCTURE ONLY (see oracle/operators.py for who may call it).

``pitsbicg`` takes the steps of Algorithm 1 (Sec. 3) in the paper's order and
notation, on the left-preconditioned system G^{-1} F Lambda = G^{-1} B of
eq. (8).  Readings of what the algorithm leaves open:

* X^0 (the "initial guess"): by default the coarse prediction G^{-1} B, the
  parareal iterate at k = 0; zero or a given array on request.
* The while test ||R^k||_{N,inf} > eps is taken relative:
  ||R^k||_{N,inf} > tol * ||R^0||_{N,inf}.
* The restart test |<R^{k+1}, R~>| <= eps0 is taken relative to
  ||R^{k+1}||_2 ||R~||_2; on restart the *new* direction is reset,
  P^{k+1} <- R^{k+1} (the listing writes P^k after P^{k+1} was formed),
  and rho is recomputed against the new shadow vector.
* Standard BiCGStab safeguards absent from the listing: exit after the half
  step when ||S^k||_{N,inf} is already below the tolerance (then
  X^{k+1} = X^k + alpha_k P^k); a vanishing <D, R~> (below
  ``breakdown_eps`` ||D||_2 ||R~||_2) triggers one restart and, if it
  vanishes again, a breakdown status; omega_k = 0 is a breakdown.

``parareal`` is the algebraic form (6): Lambda^{k+1} = Lambda^k + G^{-1}(B - F Lambda^k),
which equals the predictor-corrector (5) read as
lam_{n+1}^{k+1} = G(lam_n^{k+1}) + F(lam_n^k) - G(lam_n^k).

Matvec accounting follows Sec. 4: one application of G^{-1} F per parareal
iteration, two per PiTSBiCG iteration (plus one for the initial residual).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Union

import numpy as np

from .operators import OracleProblem, block_dot, norm2, norm_N_inf

OK = "ok"
MAXITER = "maxiter"
BREAKDOWN = "breakdown"


@dataclasses.dataclass
class SolveInfo:
    iterations: int = 0
    matvecs: int = 0
    restarts: int = 0
    status: str = OK
    r0: float = 0.0
    precond_resid: float = 0.0
    history: List[float] = dataclasses.field(default_factory=list)
    scalars: List[dict] = dataclasses.field(default_factory=list)
    R: Optional[np.ndarray] = None          # the recursively updated residual at exit


def _initial_guess(prob: OracleProblem, x0: Union[str, np.ndarray]) -> np.ndarray:
    if isinstance(x0, str):
        if x0 == "coarse":
            return prob.coarse_prediction()
        if x0 == "zero":
            return prob.zeros()
        raise ValueError(x0)
    return np.array(x0, dtype=np.float64).reshape(prob.N + 1, prob.M)


def pitsbicg(prob: OracleProblem, tol: float, eps0: float = 1e-8, max_iter: int = 1000,
             x0: Union[str, np.ndarray] = "coarse", abs_tol: Optional[float] = None,
             breakdown_eps: float = 1e-14):
    """Algorithm 1 (PiTSBiCG).  Returns (X, SolveInfo).

    ``abs_tol`` replaces the relative threshold tol * ||R^0||_{N,inf} when given.
    ``info.scalars`` records alpha, omega, beta, rho per iteration.
    """
    info = SolveInfo()
    B = prob.rhs()
    X = _initial_guess(prob, x0)
    R = prob.sweep_Ginv(B - prob.apply_F(X))          # R^0 = G^{-1}(B - F X^0)
    info.matvecs += 1
    Rt = R.copy()                                      # R~ = R^0
    P = R.copy()                                       # P^0 = R^0
    rho = block_dot(R, Rt)
    info.r0 = norm_N_inf(R)
    thresh = abs_tol if abs_tol is not None else tol * info.r0
    rnorm = info.r0
    info.history.append(rnorm)
    k = 0
    just_restarted = False
    while rnorm > thresh:
        if k >= max_iter:
            info.status = MAXITER
            break
        D = prob.apply_GinvF(P)                        # D^k = G^{-1} F P^k
        info.matvecs += 1
        sigma = block_dot(D, Rt)
        if abs(sigma) <= breakdown_eps * norm2(D) * norm2(Rt):
            if just_restarted:
                info.status = BREAKDOWN
                break
            Rt = R.copy()
            P = R.copy()
            rho = block_dot(R, Rt)
            info.restarts += 1
            just_restarted = True
            continue
        just_restarted = False
        alpha = rho / sigma                            # alpha_k = <R^k,R~>/<D^k,R~>
        S = R - alpha * D                              # S^k = R^k - alpha_k D^k
        snorm = norm_N_inf(S)
        if snorm <= thresh:                            # half-step exit
            X = X + alpha * P
            R = S
            rnorm = snorm
            k += 1
            info.scalars.append({"alpha": alpha, "omega": 0.0, "beta": 0.0, "rho": rho})
            info.history.append(rnorm)
            break
        K = prob.apply_GinvF(S)                        # K^k = G^{-1} F S^k
        info.matvecs += 1
        kk = block_dot(K, K)
        omega = block_dot(K, S) / kk                   # omega_k = <K,S>/<K,K>
        if omega == 0.0:
            info.status = BREAKDOWN
            break
        X = X + alpha * P + omega * S                  # X^{k+1}
        R_new = S - omega * K                          # R^{k+1} = S^k - omega_k K^k
        rho_new = block_dot(R_new, Rt)
        beta = (alpha / omega) * (rho_new / rho)       # beta_k
        P = R_new + beta * (P - omega * D)             # P^{k+1}
        if abs(rho_new) <= eps0 * norm2(R_new) * norm2(Rt):   # restart on small rho
            Rt = R_new.copy()
            P = R_new.copy()
            rho_new = block_dot(R_new, Rt)
            info.restarts += 1
        info.scalars.append({"alpha": alpha, "omega": omega, "beta": beta, "rho": rho})
        R = R_new
        rho = rho_new
        k += 1
        rnorm = norm_N_inf(R)
        info.history.append(rnorm)
    info.iterations = k
    info.precond_resid = rnorm
    info.R = R
    return X, info


def parareal(prob: OracleProblem, kmax: int, tol: float = 0.0,
             x0: Union[str, np.ndarray] = "coarse", abs_tol: Optional[float] = None):
    """Parareal in algebraic form (6).  Returns (X, SolveInfo).

    Stops when ||G^{-1}(B - F X^k)||_{N,inf} <= tol * r0 (the same preconditioned
    residual as PiTSBiCG's) or after ``kmax`` corrections.
    """
    info = SolveInfo()
    X = _initial_guess(prob, x0)
    B = prob.rhs()
    k = 0
    while True:
        R = prob.sweep_Ginv(B - prob.apply_F(X))
        info.matvecs += 1
        rnorm = norm_N_inf(R)
        if k == 0:
            info.r0 = rnorm
        info.history.append(rnorm)
        thresh = abs_tol if abs_tol is not None else tol * info.r0
        if rnorm <= thresh:
            break
        if k >= kmax:
            info.status = MAXITER if tol > 0 or abs_tol is not None else OK
            break
        X = X + R                                      # Lambda^{k+1} = Lambda^k + G^{-1}(B - F Lambda^k)
        k += 1
    info.iterations = k
    info.precond_resid = rnorm
    return X, info
