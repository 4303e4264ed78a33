"""EIFE-linear time stepping (Eq. (1-7)) and Parareal Algorithm 1, per mode.

Test infrastructure only (see ``oracle/__init__``).

After the simultaneous diagonalisation (Sec. 2.3) the semi-discrete system
Eq. (1-5) decouples into scalar ODEs c_J' = -lam_J c_J + ghat_J(t) with
ghat = the modal coefficients of P_h f(t).  On each mode the EIFE-linear
step Eq. (1-7) with step tau reads

    c <- e^{-lam tau} c + tau * sum_i b_i(-lam tau) ghat(t + c_i tau),

with b_i from Eq. (3-12).  The coarse propagator G is one such step of
size dT with the p coarse nodes; the fine propagator F^M is M steps of size
dt = dT/M with the q fine nodes (Sec. 2.3).  ``parareal`` runs Algorithm 1
as printed: a sequential coarse sweep, then per iteration the fine
propagator from every slice start, then the sequential correction
Eq. (Parareal), recomputing G at the previous iterate.

Stopping rule (the paper leaves it open): the relative residual
r_k = sqrt(sum_{n=1}^N ||U^{n,(k)} - U^{n,(k-1)}||_0^2) / sqrt(sum_n ||U^{n,(k)}||_0^2)
<= tol, or k = N (Theorem 4.3 makes k = N exact).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Optional

import numpy as np

from . import dirichlet, fem, quadrature
from .phi import b_weights


class ModalSystem:
    """The decoupled modal ODE system of one problem on a set of modes.

    basis:          'closed_form' (DST-I eigenpairs) or 'dense' (generalized
                    eigensolve, tiny grids).
    forcing_route:  'separable' evaluates P_h f of a separable source as the
                    outer product of 1D projections; 'full' assembles the
                    d-D consistent load by element quadrature at every stage
                    time and transforms it.
    modes:          optional flat indices of a subset of modes (closed-form
                    basis, separable route only).  Modes are independent, so
                    results on a subset equal the full run restricted to it.
    """

    def __init__(self, prob, basis: str = "closed_form", forcing_route: str = "separable",
                 modes: Optional[np.ndarray] = None):
        self.prob = prob
        self.forcing_route = forcing_route
        n, box, qp = prob.n, prob.box, prob.quad_pts
        self.periodic = tuple(getattr(prob, "periodic", ())) + (False,) * (prob.d - len(getattr(prob, "periodic", ())))
        if any(self.periodic) and getattr(prob, "boundary", ()):
            raise ValueError("Dirichlet data with periodic axes are not supported")
        if basis == "closed_form":
            self.basis = fem.ClosedFormBasis(n, box, prob.D, self.periodic)
        elif basis == "dense":
            self.basis = fem.DenseBasis(n, box, prob.D, self.periodic)
        else:
            raise ValueError(basis)
        self.modes = None if modes is None else np.asarray(modes, dtype=np.int64)
        if self.modes is not None and (basis != "closed_form" or forcing_route != "separable"):
            raise ValueError("mode subsets need the closed-form basis and the separable route")

        lam = np.asarray(self.basis.lam, dtype=np.float64).reshape(-1)
        w = np.asarray(self.basis.norm2_weights(), dtype=np.float64).reshape(-1)
        self.lam = lam if self.modes is None else lam[self.modes]
        self.norm_w = w if self.modes is None else w[self.modes]

        if forcing_route == "separable":
            if any(quadrature.is_time_dependent(f) for term in prob.forcing for f in term.factors):
                raise ValueError("time-dependent spatial factors need forcing_route='full'")
            self._P = [self._separable_modal(term) for term in prob.forcing]
            # u0 = sum of its terms; no terms is the zero function (P_h 0 = 0)
            self.c0 = np.zeros_like(self.lam) + sum(term.amp * self._separable_modal(term) for term in prob.u0)
        elif forcing_route == "full":
            self._P = None
            F0 = quadrature.load_full(prob.u0, None, n, box, qp, self.periodic)
            self.c0 = np.asarray(self.basis.to_modal_from_load(F0)).reshape(-1)
        else:
            raise ValueError(forcing_route)
        # non-homogeneous Dirichlet data: w = u_h - I_h g, w(t0) = P_h(u0 - I_h g(t0))
        self.lift = dirichlet.DirichletLift(prob) if getattr(prob, "boundary", ()) else None
        if self.lift is not None:
            self.c0 = self.c0 - self._restrict(self.basis.to_modal_from_load(self.lift.lift_load(prob.t0)))

    def _restrict(self, c: np.ndarray) -> np.ndarray:
        c = np.asarray(c).reshape(-1)
        return c if self.modes is None else c[self.modes]

    def _separable_modal(self, term) -> np.ndarray:
        """Modal coefficients of P_h of the spatial part of one separable term."""
        prob = self.prob
        loads = quadrature.separable_load_factors(term, prob.n, prob.box, prob.quad_pts, self.periodic)
        if isinstance(self.basis, fem.ClosedFormBasis):
            axis = [self.basis.axis_modal_factor(a, loads[a]) for a in range(prob.d)]
            if self.modes is None:
                return fem.outer_all(axis).reshape(-1)
            idx = np.unravel_index(self.modes, prob.n)
            out = np.ones(len(self.modes))
            for a in range(prob.d):
                out = out * axis[a][idx[a]]
            return out
        F = fem.outer_all(loads)
        return np.asarray(self.basis.to_modal_from_load(F)).reshape(-1)

    def ghat(self, t: float) -> np.ndarray:
        """Modal coefficients of P_h f(t) (plus the lifting's extra load under Dirichlet data)."""
        if self.forcing_route == "separable":
            out = np.zeros_like(self.lam)
            for term, P in zip(self.prob.forcing, self._P):
                out = out + (term.amp * quadrature.eval_time(term, t)) * P
        else:
            prob = self.prob
            F = quadrature.load_full(prob.forcing, t, prob.n, prob.box, prob.quad_pts, self.periodic)
            out = np.asarray(self.basis.to_modal_from_load(F)).reshape(-1)
        if self.lift is not None:
            out = out + self._restrict(self.basis.to_modal_from_load(self.lift.extra_load(t)))
        return out

    def solution_nodal(self, c: np.ndarray, t: float) -> np.ndarray:
        """Interior nodal values of u_h = w + I_h g at time t for the modal state c of w."""
        u = self.to_nodal(c)
        return u if self.lift is None else u + self.lift.interior(t)

    def norm(self, c: np.ndarray) -> float:
        """||v||_0 of the FE function with modal coefficients c."""
        return float(np.sqrt(np.sum(self.norm_w * c * c)))

    def to_nodal(self, c: np.ndarray) -> np.ndarray:
        if self.modes is not None:
            raise ValueError("nodal values need all modes")
        return self.basis.to_nodal(c.reshape(self.prob.n) if isinstance(self.basis, fem.ClosedFormBasis) else c)


class Stepper:
    """E = e^{-lam tau} and b_i(-lam tau) for one step size and one node set."""

    def __init__(self, lam: np.ndarray, tau: float, nodes):
        self.tau = float(tau)
        self.nodes = tuple(float(c) for c in nodes)
        z = -lam * self.tau
        self.E = np.exp(z)
        self.b = b_weights(z, self.nodes)

    def step(self, c: np.ndarray, t: float, ghat: Callable[[float], np.ndarray]) -> np.ndarray:
        """One EIFE-linear step, Eq. (1-7), from time t."""
        acc = np.zeros_like(c)
        for i, ci in enumerate(self.nodes):
            acc = acc + self.b[i] * ghat(t + ci * self.tau)
        return self.E * c + self.tau * acc


def sequential_eife(sys: ModalSystem, n_steps: int, nodes, c0: Optional[np.ndarray] = None,
                    t_start: Optional[float] = None, duration: Optional[float] = None) -> np.ndarray:
    """EIFE-linear with n_steps uniform steps over [t_start, t_start + duration]."""
    prob = sys.prob
    t_start = prob.t0 if t_start is None else t_start
    duration = prob.T if duration is None else duration
    tau = duration / n_steps
    st = Stepper(sys.lam, tau, nodes)
    c = sys.c0.copy() if c0 is None else c0.copy()
    for l in range(n_steps):
        c = st.step(c, t_start + l * tau, sys.ghat)
    return c


def sequential_fine(sys: ModalSystem) -> List[np.ndarray]:
    """Fine EIFE run sequentially over all N*M fine steps; returns the N+1 slice values."""
    prob = sys.prob
    dT = prob.T / prob.N
    dt = dT / prob.M
    st = Stepper(sys.lam, dt, prob.fine_nodes)
    out = [sys.c0.copy()]
    c = sys.c0.copy()
    for n in range(prob.N):
        Tn = prob.t0 + n * dT
        for m in range(prob.M):
            c = st.step(c, Tn + m * dt, sys.ghat)
        out.append(c.copy())
    return out


@dataclass
class PararealResult:
    U: List[np.ndarray]            # final iterate, N+1 slice values
    history: List[List[np.ndarray]]  # iterates U^{(0)}, U^{(1)}, ...
    residuals: List[float]         # r_k for k = 1, 2, ...
    k: int                         # iterations performed


class Propagators:
    """G and F^M of Sec. 2.3 on one modal system."""

    def __init__(self, sys: ModalSystem):
        p = sys.prob
        self.sys = sys
        self.dT = p.T / p.N
        self.dt = self.dT / p.M
        self.coarse = Stepper(sys.lam, self.dT, p.coarse_nodes)
        self.fine = Stepper(sys.lam, self.dt, p.fine_nodes)

    def T(self, n: int) -> float:
        return self.sys.prob.t0 + n * self.dT

    def G(self, v: np.ndarray, n: int) -> np.ndarray:
        return self.coarse.step(v, self.T(n), self.sys.ghat)

    def FM(self, v: np.ndarray, n: int) -> np.ndarray:
        c = v.copy()
        for m in range(self.sys.prob.M):
            c = self.fine.step(c, self.T(n) + m * self.dt, self.sys.ghat)
        return c


def parareal(sys: ModalSystem, tol: float = 0.0, k_max: Optional[int] = None,
             keep_history: bool = True) -> PararealResult:
    """Algorithm 1 (PEIFE-linear) with the residual stopping rule above."""
    N = sys.prob.N
    k_max = N if k_max is None else min(k_max, N)
    prop = Propagators(sys)
    U = [sys.c0.copy()]
    for n in range(N):                          # coarse sweep, k = 0
        U.append(prop.G(U[n], n))
    history = [list(U)] if keep_history else []
    residuals: List[float] = []
    k = 0
    while k < k_max:
        Fbar = [prop.FM(U[n], n) for n in range(N)]          # parallel in n
        Unew = [sys.c0.copy()]
        for n in range(N):                                    # sequential correction
            Unew.append(prop.G(Unew[n], n) + Fbar[n] - prop.G(U[n], n))
        num = sum(sys.norm(Unew[n] - U[n]) ** 2 for n in range(1, N + 1))
        den = sum(sys.norm(Unew[n]) ** 2 for n in range(1, N + 1))
        r = float(np.sqrt(num) / np.sqrt(den)) if den > 0 else float(np.sqrt(num))
        residuals.append(r)
        U = Unew
        k += 1
        if keep_history:
            history.append(list(U))
        if r <= tol:
            break
    return PararealResult(U, history, residuals, k)


def rel_l2(a: np.ndarray, b: np.ndarray, weights: np.ndarray) -> float:
    """||a - b||_0 / ||b||_0 for modal coefficient arrays with norm weights muM."""
    num = np.sqrt(np.sum(weights * (a - b) ** 2))
    den = np.sqrt(np.sum(weights * b * b))
    return float(num / den) if den > 0 else float(num)
