"""Two-level PFASST with spectral coarsening (Sections 5.1.2, 5.2, 5.3; Algorithm 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The n_ts "processors" of the paper are emulated by a plain sequential loop
over time slices in rank order; a send is a copy into the receiver's array.

* Space restriction D (Eq. "space_restriction"): keep the coefficients with
  n <= T_c (and hence m <= T_c) of each field; space interpolation is its
  transpose, zero-padding.
* Time restriction Pi_f^c (Eq. "time_restriction"): Lagrange polynomials of the
  fine nodes evaluated at the coarse nodes; time interpolation Pi_c^f
  (Eq. "time_interpolation"): Lagrange polynomials of the coarse nodes at the
  fine nodes.
* FAS (Eq. "tau_term_level_l+1" with tau_f = 0): tau_c = A_c(R Theta_f) -
  R A_f(Theta_f) = dt [R (Q_f F_f) - Q_c F_c(R Theta_f)]; the Theta terms cancel
  because R is linear.  tau_c is cumulative from t^n, as the node update of
  Eq. "modified_update_equation_sdcq_discrete_form" adds it to Theta_0.
* Predictor (Section 5.2.1): the initial value is broadcast and restricted;
  in round j = 0..n_ts-1 every slice n >= j takes as its coarse initial value
  the end value slice n-1 had after round j-1 (round 0: the broadcast value),
  refreshes its node-0 right-hand side and performs one coarse sweep; slice
  n thus sweeps n+1 times.  The coarse result is brought to the fine level
  as an increment (coarse minus the restricted broadcast value) added to the
  broadcast fine value at every node -- the paper defers the details of
  this step to Emmett & Minion 2012; using an increment keeps the fine modes
  of the initial value, the same way Step D does.  Fine right-hand sides
  are then evaluated at all nodes.
* Iteration (Algorithm 1): A) fine sweep; stop here on the last iteration.
  B) restrict, evaluate coarse F at every coarse node, save Theta~_c, F~_c,
  compute tau_c.  C) slices in order: receive the new coarse initial value
  from slice n-1 (slice 0 keeps its own), refresh node-0 F, coarse sweep
  with tau.  D) add interpolated increments Theta_c - Theta~_c,
  F_{I,c} - F~_{I,c}, F_{E,c} - F~_{E,c} at all fine nodes; then the fine
  initial value of slice n >= 1 becomes the value slice n-1 sent in Step A
  plus the interpolated node-0 coarse increment (last line of Algorithm 1,
  read with m = 0 as the text says).  The increment is taken against the
  restriction of the value just received, i.e. new coarse initial value
  minus R(received fine value), which equals slice n-1's coarse increment at
  its last node.  Taking it literally against the saved Theta~_c of the
  slice's old initial value makes the iteration diverge even with alpha = 1
  (error grows with every iteration once n_ts > 1), so that reading is
  rejected.  Finally the fine right-hand side at node 0 is re-evaluated
  (last term of the iteration cost in Section 5.5).

The steps that are independent across slices go through ``_each``, which
either loops here or hands the same level method to worker processes
(``oracle.pool``); the arithmetic is the same either way.

Pins (tests/test_oracle_pfasst.py): R o P = identity; nested Lobatto time
restriction is injection; the FAS invariant (a coarse sweep with tau leaves
the restriction of a fine collocation solution unchanged); with enough
iterations PFASST converges to the serial collocation solution of every
slice, for alpha = 1 and alpha < 1; the predictor's rounds equal the
slice-by-slice statement (slice n sweeps n + 1 times, each time from its
predecessor's value of the previous round); the worker pool changes no bit.
"""
from __future__ import annotations

import numpy as np

from .sdc import SDCLevel, lagrange_matrix


def restrict_space(x: np.ndarray, Lc: int) -> np.ndarray:
    return x[..., :Lc, :Lc].copy()


def interpolate_space(x: np.ndarray, Lf: int) -> np.ndarray:
    out = np.zeros(x.shape[:-2] + (Lf, Lf), dtype=np.complex128)
    Lc = x.shape[-1]
    out[..., :Lc, :Lc] = x
    return out


class PFASST:
    """``pool`` (optional): an ``oracle.pool.SlicePool`` whose levels "f" and
    "c" were built from ``fine.args`` and ``coarse.args``; the per-slice
    independent steps then run in its worker processes (same arithmetic)."""

    def __init__(self, fine: SDCLevel, coarse: SDCLevel, n_ts: int, pool=None):
        self.f, self.c, self.n_ts = fine, coarse, n_ts
        self.Lf, self.Lc = fine.T + 1, coarse.T + 1
        self.R_t = lagrange_matrix(fine.tau, coarse.tau)     # (Mc+1, Mf+1)
        self.P_t = lagrange_matrix(coarse.tau, fine.tau)     # (Mf+1, Mc+1)
        self.pool = pool

    def _each(self, level: str, method: str, arg_tuples: list) -> list:
        """[getattr(level, method)(*a) for a in arg_tuples], slices in order;
        the calls are independent of one another."""
        if self.pool is None or len(arg_tuples) < 2:
            lvl = self.f if level == "f" else self.c
            return [getattr(lvl, method)(*a) for a in arg_tuples]
        return self.pool.run(level, method, arg_tuples)

    # ---- transfer operators on space-time vectors [nodes, 3, L, L] ----
    def restrict(self, x_f: np.ndarray) -> np.ndarray:
        xt = np.einsum("ij,j...->i...", self.R_t, x_f)
        return restrict_space(xt, self.Lc)

    def interpolate(self, x_c: np.ndarray) -> np.ndarray:
        xs = interpolate_space(x_c, self.Lf)
        return np.einsum("ij,j...->i...", self.P_t, xs)

    def fas(self, FE_f, FI_f, FE_c, FI_c) -> np.ndarray:
        QF_f = np.einsum("ij,j...->i...", self.f.Q, FE_f + FI_f)
        QF_c = np.einsum("ij,j...->i...", self.c.Q, FE_c + FI_c)
        return self.f.dt * self.restrict(QF_f) - self.c.dt * QF_c

    # ---- predictor (Section 5.2.1) ----
    def predict(self, theta0: np.ndarray) -> None:
        n_ts, Mc = self.n_ts, self.c.M
        th0_c = restrict_space(theta0, self.Lc)
        self.th_c = np.repeat(np.repeat(th0_c[None], Mc + 1, 0)[None], n_ts, 0)
        fe0, fi0 = self.c.eval_f(th0_c)
        self.FE_c = np.repeat(np.repeat(fe0[None], Mc + 1, 0)[None], n_ts, 0)
        self.FI_c = np.repeat(np.repeat(fi0[None], Mc + 1, 0)[None], n_ts, 0)
        base_c = self.th_c.copy()
        for j in range(n_ts):
            ends = self.th_c[:, Mc].copy()           # values after round j-1
            recv = [n for n in range(max(j, 1), n_ts)] if j > 0 else []
            for n in recv:
                self.th_c[n, 0] = ends[n - 1]
            for n, (fe, fi) in zip(recv, self._each("c", "eval_f", [(self.th_c[n, 0],) for n in recv])):
                self.FE_c[n, 0], self.FI_c[n, 0] = fe, fi
            swept = self._each("c", "sweep", [(self.th_c[n], self.FE_c[n], self.FI_c[n]) for n in range(j, n_ts)])
            for n, (th, fe, fi) in zip(range(j, n_ts), swept):
                self.th_c[n], self.FE_c[n], self.FI_c[n] = th, fe, fi
        Mf = self.f.M
        self.th_f = np.empty((n_ts, Mf + 1) + theta0.shape, dtype=np.complex128)
        self.FE_f = np.empty_like(self.th_f)
        self.FI_f = np.empty_like(self.th_f)
        for n in range(n_ts):
            self.th_f[n] = theta0[None] + self.interpolate(self.th_c[n] - base_c[n])
        for n, (fe, fi) in enumerate(self._each("f", "eval_nodes", [(self.th_f[n],) for n in range(n_ts)])):
            self.FE_f[n], self.FI_f[n] = fe, fi

    # ---- one iteration of Algorithm 1 ----
    def iteration(self, last: bool = False) -> None:
        n_ts, Mf, Mc = self.n_ts, self.f.M, self.c.M
        # A) fine sweeps (parallel across slices)
        swept = self._each("f", "sweep", [(self.th_f[n], self.FE_f[n], self.FI_f[n]) for n in range(n_ts)])
        for n, (th, fe, fi) in enumerate(swept):
            self.th_f[n], self.FE_f[n], self.FI_f[n] = th, fe, fi
        if last:
            return
        sent_f = self.th_f[:, Mf].copy()
        # B) restrict, re-evaluate, save, FAS
        tau = np.empty((n_ts, Mc + 1) + self.th_c.shape[2:], dtype=np.complex128)
        for n in range(n_ts):
            self.th_c[n] = self.restrict(self.th_f[n])
        for n, (fe, fi) in enumerate(self._each("c", "eval_nodes", [(self.th_c[n],) for n in range(n_ts)])):
            self.FE_c[n], self.FI_c[n] = fe, fi
            tau[n] = self.fas(self.FE_f[n], self.FI_f[n], self.FE_c[n], self.FI_c[n])
        th_c_saved = self.th_c.copy()
        FE_c_saved = self.FE_c.copy()
        FI_c_saved = self.FI_c.copy()
        # C) serial coarse chain
        for n in range(n_ts):
            if n > 0:
                self.th_c[n, 0] = self.th_c[n - 1, Mc]
                self.FE_c[n, 0], self.FI_c[n, 0] = self.c.eval_f(self.th_c[n, 0])
            self.th_c[n], self.FE_c[n], self.FI_c[n] = self.c.sweep(
                self.th_c[n], self.FE_c[n], self.FI_c[n], tau[n])
        # D) interpolate increments, new fine initial values, refresh node 0
        for n in range(n_ts):
            d_th = self.interpolate(self.th_c[n] - th_c_saved[n])
            self.th_f[n] += d_th
            self.FI_f[n] += self.interpolate(self.FI_c[n] - FI_c_saved[n])
            self.FE_f[n] += self.interpolate(self.FE_c[n] - FE_c_saved[n])
            if n > 0:
                received = sent_f[n - 1]
                self.th_f[n, 0] = received + interpolate_space(
                    self.th_c[n, 0] - restrict_space(received, self.Lc), self.Lf)
        for n, (fe, fi) in enumerate(self._each("f", "eval_f", [(self.th_f[n, 0],) for n in range(n_ts)])):
            self.FE_f[n, 0], self.FI_f[n, 0] = fe, fi

    def run(self, theta0: np.ndarray, n_iter: int) -> np.ndarray:
        """Predictor + n_iter iterations (the last one is Step A only);
        returns the end values [n_ts, 3, L, L] of every slice."""
        self.predict(theta0)
        for k in range(n_iter):
            self.iteration(last=(k == n_iter - 1))
        return self.th_f[:, self.f.M].copy()
