"""Plain FP64 CPU oracle of the windowed regularized LBM-LES and its discrete adjoint.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA path.  It is slow on purpose: every step is the
paper's definition written out over whole numpy arrays, with no fusion, blocking
or reordering, so that a reader can check it against the paper by eye.  Complex
input arrays are supported throughout so that complex-step derivatives of the
forward map can pin the adjoint.

What it computes, by paper reference:

* lattice, equilibrium, moments ............ Sec. 2.1.1, Eqs. 2-5
* regularized LES collision ................ Sec. 2.1.2, Eqs. 9-16
* wall / Zou-He inlet / Zou-He outlet ...... Sec. 2.1.3, Eqs. 18-21
* partial bounce-back ...................... Sec. 2.2, Eq. 23 and g(phi)
* window means and the criterion ........... Sec. 3.1, Eqs. 24-26; Eq. 42
* window objective ......................... Sec. 3.2, Eq. 27
* discrete adjoint (literal Jacobian) ...... Sec. 3.2, Eqs. 30-36
* adjoint boundary rules ................... Eqs. 37-39, here as the transpose
  of the explicit stream+boundary operator
* design sensitivity ....................... Eq. 40

Readings where the paper is silent or ambiguous (each is also listed in the
design notes):

* the carried state is the post-collision field p; step n pulls p^{n-1}
  through streaming and the boundary rules into f^n, then collides f^n into
  p^n; the initial carried field is the equilibrium at rho=1, u=0;
* the norm in Eq. 14 is |Pi| = sqrt(2 Pi:Pi), the convention of |S| under Eq. 9;
  its derivative is taken as 0 where |Pi| = 0;
* the wall rule of Eq. 19 is applied to every wall node as "an unknown
  population takes the value of its opposite"; when the opposite is unknown
  too (a corner's buried link) the population is set to its rest weight w_a;
* the interpolation parameter of g(phi) is named q here (the paper calls it
  gamma), default 0.1; the input design field gamma is the solid fraction,
  phi = 1 - gamma;
* a window of |W| steps samples f^n at the steps n0, n0+dW, ...; the objective
  source enters the adjoint at those steps with weight dW/|W| (Eq. 42);
* full-time adjoint (Sec. 4.2.3, the comparison with full-time adjoint
  optimization): the run from the initial time is one window of T steps whose
  samples start at step T - |W| (case.sample_from), so the objective is the
  mean over the final |W| steps while the adjoint is traced back to step 0;
  the weight is then dW/(T - sample_from);
* D3Q19 (beyond the paper): same collision with p,q in {x,y,z}; velocity
  inlet by the linear moving-wall bounce-back f_a = f_abar + 2 w_a rho0 c_a.u/cs^2
  with rho0 = 1; zero-gradient outlet copies the neighbour along the inward normal.

Pins: every function above is checked against closed forms, invariants, the
paper's printed adjoint boundary coefficients, complex-step derivatives and
finite differences (tests/test_oracle_*.py), with planted mistakes that must
fail them.  Parity unpinned: the absolute values of J and C_d on the
benchmark workloads' own geometries, for which the paper prints no values.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

FLUID, WALL, INLET, OUTLET_P, OUTLET_ZG = 0, 1, 2, 3, 4
OBJ_DISSIPATION, OBJ_VELOCITY_DEV, OBJ_PRESSURE, OBJ_DRAG = 0, 1, 2, 3
MON_DRAG, MON_OBJECTIVE = 0, 1

CS2 = 1.0 / 3.0          # c_s^2, Sec. 2.1.1 (c_s = sqrt(3)/3)
CS4 = CS2 * CS2


class Lattice:
    """Discrete velocities c_a, weights w_a and opposite directions."""

    def __init__(self, q: int):
        if q == 9:
            # Sec. 2.1.1, Eq. 2 (velocity order) and Eq. 4 (weights).
            c = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0),
                 (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)]
            w = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
            d = 2
        elif q == 19:
            # Standard D3Q19: rest 1/3, axis 1/18, face diagonals 1/36.
            c = [(0, 0, 0),
                 (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                 (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
                 (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
                 (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
            w = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
            d = 3
        else:
            raise ValueError("lattice must be 9 or 19")
        self.q = q
        self.d = d
        self.c3 = np.array(c, dtype=np.int64)          # (Q, 3)
        self.c = self.c3[:, :d].astype(np.float64)      # (Q, d)
        self.w = np.array(w, dtype=np.float64)
        self.opp = np.array([next(b for b in range(q) if (self.c3[b] == -self.c3[a]).all())
                             for a in range(q)])
        # Q_a,pq = c_ap c_aq - c_s^2 delta_pq  (Eq. 16)
        self.Qt = np.einsum("ap,aq->apq", self.c, self.c) - CS2 * np.eye(d)[None]


# ---------------------------------------------------------------------------
# Local (per node) operators.  Arrays: populations (Q, N); vectors (d, N).
# ---------------------------------------------------------------------------

def density(f):
    """rho = sum_a f_a (Eq. 5a)."""
    return f.sum(axis=0)


def velocity(lat, f, rho):
    """u = sum_a c_a f_a / rho (Eq. 5b)."""
    return (lat.c.T @ f) / rho


def equilibrium(lat, rho, u):
    """f^eq_a = w_a rho [1 + c.u/cs^2 + (c.u)^2/(2cs^4) - u.u/(2cs^2)] (Eq. 3)."""
    cu = lat.c @ u                                   # (Q, N)
    uu = (u * u).sum(axis=0)
    return lat.w[:, None] * rho[None] * (1.0 + cu / CS2 + cu * cu / (2 * CS4) - uu[None] / (2 * CS2))


def pi_neq(lat, f, feq):
    """Pi_pq = sum_a c_ap c_aq (f_a - f^eq_a) (Eq. 13); shape (d, d, N)."""
    return np.einsum("ap,aq,an->pqn", lat.c, lat.c, f - feq)


def pi_norm(pi):
    """|Pi| = sqrt(2 Pi:Pi), the norm that turns Eqs. 9-12 into Eq. 14."""
    return np.sqrt(2.0 * (pi * pi).sum(axis=(0, 1)))


def tau_effective(tau, cs_smag, rho, pinorm):
    """tau_eff = (tau + sqrt(tau^2 + 2 (Cs l)^2 |Pi| / (rho cs^4))) / 2 (Eq. 14), l = 1."""
    return 0.5 * (tau + np.sqrt(tau * tau + 2.0 * cs_smag ** 2 * pinorm / (rho * CS4)))


def regularized_neq(lat, pi):
    """w_a / (2 cs^4) sum_pq (c_ap c_aq - cs^2 delta_pq) Pi_pq (the bracket of Eq. 16)."""
    return lat.w[:, None] / (2 * CS4) * np.einsum("apq,pqn->an", lat.Qt, pi)


def g_of_phi(phi, q, g_max):
    """g(phi) = g_max (1 - phi (1 + q) / (phi + q)), g_max = 1/2 in Sec. 2.2."""
    return g_max * (1.0 - phi * (1.0 + q) / (phi + q))


def dg_dphi(phi, q, g_max):
    """Derivative of g(phi): -g_max q (1 + q) / (phi + q)^2."""
    return -g_max * q * (1.0 + q) / (phi + q) ** 2


def collide(lat, f, tau, cs_smag):
    """Regularized LES collision h = f^eq + (1 - 1/tau_eff) * reg. neq (Eq. 16).

    Returns h and the intermediate quantities the adjoint and objectives need.
    """
    rho = density(f)
    u = velocity(lat, f, rho)
    feq = equilibrium(lat, rho, u)
    pi = pi_neq(lat, f, feq)
    pn = pi_norm(pi)
    te = tau_effective(tau, cs_smag, rho, pn)
    hneq = regularized_neq(lat, pi)
    h = feq + (1.0 - 1.0 / te)[None] * hneq
    return h, dict(rho=rho, u=u, feq=feq, pi=pi, pinorm=pn, tau_eff=te, hneq=hneq)


def blend(lat, h, g):
    """Partial bounce-back: p_a = h_a + F_a, F_a = g (h_abar - h_a) (Eq. 23)."""
    return h + g[None] * (h[lat.opp] - h)


# ---------------------------------------------------------------------------
# Streaming and boundary rules as one explicit affine operator f = S p + s0.
# ---------------------------------------------------------------------------

class _Affine:
    """A population written as sum_k coef_k * p[col_k] + const."""

    def __init__(self, terms=None, const=0.0):
        self.t = dict(terms or {})
        self.k = const

    def __add__(self, o):
        r = _Affine(self.t, self.k)
        for c, v in o.t.items():
            r.t[c] = r.t.get(c, 0.0) + v
        r.k += o.k
        return r

    def __sub__(self, o):
        return self + o * -1.0

    def __mul__(self, s):
        return _Affine({c: v * s for c, v in self.t.items()}, self.k * s)

    __rmul__ = __mul__


class Problem:
    """Geometry, parameters and the stream+boundary operator of one case.

    ``case`` is any object with the attributes of ``inputs.Case`` (lattice, nx,
    ny, nz, tau, cs_smag, node_class, gamma, inlet_u, obj_weights, obj_kind,
    obj_uref, q_interp, g_max, rho_out, periodic, monitor_kind, monitor_u,
    monitor_l, window_len, sample_every, sample_from, conv_tol).
    """

    def __init__(self, case):
        self.case = case
        self.lat = Lattice(case.lattice)
        self.nx, self.ny, self.nz = case.nx, case.ny, case.nz
        self.n = self.nx * self.ny * self.nz
        self.tau = float(case.tau)
        self.cs = float(case.cs_smag)
        self.cls = np.asarray(case.node_class, np.uint8).reshape(-1)
        self.w_obj = np.asarray(case.obj_weights, np.float64).reshape(-1)
        self.S, self.s0 = self._build_stream_bc()

    # -- geometry ----------------------------------------------------------
    def _coords(self):
        i = np.arange(self.n)
        return i % self.nx, (i // self.nx) % self.ny, i // (self.nx * self.ny)

    def _source(self, x, y, z, a):
        """Node that streams into (x,y,z) along c_a: (x,y,z) - c_a, or -1 if outside."""
        dims = (self.nx, self.ny, self.nz)
        per = self.case.periodic
        cx, cy, cz = self.lat.c3[a]
        s = [x - cx, y - cy, z - cz]
        ok = np.ones(np.shape(x), bool)
        for k in range(3):
            if per[k]:
                s[k] = np.mod(s[k], dims[k])
            else:
                ok &= (s[k] >= 0) & (s[k] < dims[k])
        idx = s[0] + self.nx * (s[1] + self.ny * s[2])
        return np.where(ok, idx, -1)

    def _build_stream_bc(self):
        """Streaming (Eq. 7) plus the boundary rules (Eqs. 19-21) as f = S p + s0."""
        lat, n, q = self.lat, self.n, self.lat.q
        x, y, z = self._coords()
        src = np.stack([self._source(x, y, z, a) for a in range(q)])     # (Q, N)
        known = src >= 0
        rows, cols, vals = [], [], []
        s0 = np.zeros(q * n)
        for a in range(q):
            m = known[a]
            rows.append(a * n + np.nonzero(m)[0])
            cols.append(a * n + src[a][m])
            vals.append(np.ones(m.sum()))
        bnodes = np.nonzero(~known.all(axis=0))[0]
        for i in bnodes:
            unk = [a for a in range(q) if not known[a, i]]
            fk = {a: _Affine({a * n + src[a, i]: 1.0}) for a in range(q) if known[a, i]}
            fill = self._boundary_rule(int(i), unk, fk, src)
            for a in unk:
                e = fill[a]
                for col, v in e.t.items():
                    rows.append(np.array([a * n + i]))
                    cols.append(np.array([col]))
                    vals.append(np.array([v]))
                s0[a * n + i] += e.k
        S = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(q * n, q * n))
        S.sum_duplicates()
        return S, s0

    def _boundary_rule(self, i, unk, fk, src):
        """Affine expressions of the unknown populations of boundary node i."""
        lat, case = self.lat, self.case
        kind = int(self.cls[i])
        x = i % self.nx
        j = i // self.nx                              # (y, z) face index of the x=0 face
        opp = lat.opp
        if kind == FLUID:
            raise ValueError(f"node {i} has unknown populations but class FLUID")
        if kind == WALL:
            # Eq. 19 applied generically: unknown f_a = f_abar; buried links -> w_a.
            return {a: (fk[opp[a]] if opp[a] in fk else _Affine(const=lat.w[a])) for a in unk}
        if kind == INLET:
            u0 = float(case.inlet_u.reshape(-1)[j])
            if x != 0:
                raise ValueError("inlet nodes must lie on the x=0 face")
            if lat.q == 9:
                if sorted(unk) != [1, 5, 8]:
                    raise ValueError(f"Zou-He inlet node {i} has unknowns {unk}")
                # Eq. 20
                rho = (fk[0] + fk[2] + fk[4] + 2.0 * (fk[3] + fk[6] + fk[7])) * (1.0 / (1.0 - u0))
                return {1: fk[3] + rho * (2.0 / 3.0 * u0),
                        5: fk[7] + (fk[4] - fk[2]) * 0.5 + rho * (u0 / 6.0),
                        8: fk[6] + (fk[2] - fk[4]) * 0.5 + rho * (u0 / 6.0)}
            out = {}
            for a in unk:
                if lat.c3[a][0] != 1 or opp[a] not in fk:
                    raise ValueError(f"velocity inlet node {i} has unknowns {unk}")
                out[a] = fk[opp[a]] + _Affine(const=2.0 * lat.w[a] * 1.0 * lat.c3[a][0] * u0 / CS2)
            return out
        if kind == OUTLET_P:
            if lat.q != 9 or x != self.nx - 1 or sorted(unk) != [3, 6, 7]:
                raise ValueError(f"Zou-He outlet node {i} has unknowns {unk}")
            r0 = float(case.rho_out)
            # Eq. 21
            u = (fk[0] + fk[2] + fk[4] + 2.0 * (fk[1] + fk[5] + fk[8])) * (1.0 / r0) + _Affine(const=-1.0)
            return {3: fk[1] - u * (2.0 / 3.0 * r0),
                    6: fk[8] + (fk[4] - fk[2]) * 0.5 - u * (r0 / 6.0),
                    7: fk[5] + (fk[2] - fk[4]) * 0.5 - u * (r0 / 6.0)}
        if kind == OUTLET_ZG:
            # f_a(i) = f_a(i + n_in) after streaming, n_in the inward x normal.
            if x == self.nx - 1:
                nb = i - 1
            elif x == 0:
                nb = i + 1
            else:
                raise ValueError("zero-gradient outlet nodes must lie on an x face")
            out = {}
            for a in unk:
                if lat.c3[a][0] == 0 or src[a, nb] < 0:
                    raise ValueError(f"zero-gradient outlet node {i} has unknowns {unk}")
                out[a] = _Affine({a * self.n + src[a, nb]: 1.0})
            return out
        raise ValueError(f"unknown node class {kind}")

    # -- design ------------------------------------------------------------
    def phi(self, gamma=None):
        g = self.case.gamma if gamma is None else gamma
        return 1.0 - np.asarray(g).reshape(-1)

    def g(self, gamma=None):
        return g_of_phi(self.phi(gamma), self.case.q_interp, self.case.g_max)

    # -- one time step -------------------------------------------------------
    def stream(self, p):
        """f^n = S p^{n-1} + s0 (streaming and boundary completion)."""
        q, n = self.lat.q, self.n
        return (self.S @ p.reshape(q * n) + self.s0).reshape(q, n)

    def stream_adjoint(self, b):
        """a^{n-1} = S^T b^n (adjoint streaming, Eq. 36, with the boundary
        rules of Eqs. 37-39 as the transpose of the forward ones)."""
        q, n = self.lat.q, self.n
        return (self.S.T @ b.reshape(q * n)).reshape(q, n)

    def step(self, p, g):
        """One step: f^n = S p^{n-1}; h = collide(f^n); p^n = blend(h)."""
        f = self.stream(p)
        h, aux = collide(self.lat, f, self.tau, self.cs)
        return f, h, blend(self.lat, h, g), aux

    def initial_state(self, dtype=np.float64):
        """Carried field at rest: f^eq(rho=1, u=0) = w_a at every node (Eq. 18)."""
        return np.repeat(self.lat.w[:, None], self.n, axis=1).astype(dtype)

    # -- objective and monitor -------------------------------------------------
    def local_objective(self, f, h, aux, g):
        """Per-node integrand psi_i of j = sum_i w_i psi_i."""
        c = self.case
        k = int(c.obj_kind)
        if k == OBJ_DISSIPATION:
            pp = (aux["pi"] * aux["pi"]).sum(axis=(0, 1))
            te = aux["tau_eff"]
            return (te - 0.5) * pp / (2.0 * aux["rho"] * CS2 * te * te)
        if k == OBJ_VELOCITY_DEV:
            du = aux["u"] - np.asarray(c.obj_uref, np.float64)[: self.lat.d, None]
            return (du * du).sum(axis=0)
        if k == OBJ_PRESSURE:
            return CS2 * aux["rho"]
        if k == OBJ_DRAG:
            return self.drag_density(h, g)
        raise ValueError("objective kind")

    def drag_density(self, h, g):
        """sum_a c_xa F_a at every node (Eq. 44 integrand), F from Eq. 23."""
        F = g[None] * (h[self.lat.opp] - h)
        return self.lat.c[:, 0] @ F

    def sample(self, f, h, aux, g):
        """Objective j(t) and monitored quantity at one sampling instant."""
        psi = self.local_objective(f, h, aux, g)
        j = (self.w_obj * psi).sum()
        if int(self.case.monitor_kind) == MON_DRAG:
            c = self.case
            mon = self.drag_density(h, g).sum() / (0.5 * c.rho_out * c.monitor_u ** 2 * c.monitor_l)
        else:
            mon = j
        return j, mon

    # -- windows -------------------------------------------------------------
    def run_window(self, p_start, gamma=None, store=True):
        """One window of |W| steps (Alg. 1 inner loop).

        Returns the final carried field, the sampled means (Eq. 42) of the
        objective and the monitor, and (if store) the carried fields
        p^{n0-1} ... p^{n0+|W|-1} of the window.
        """
        W = int(self.case.window_len)
        g = self.g(gamma)
        p = p_start
        traj = [p] if store else None
        js, ms = [], []
        for k in range(W):
            f, h, p, aux = self.step(p, g)
            if self.sampled(k):
                j, m = self.sample(f, h, aux, g)
                js.append(j)
                ms.append(m)
            if store:
                traj.append(p)
        weight = self.sample_weight()
        return p, weight * sum(js), weight * sum(ms), traj

    def sampled(self, k):
        """Is step k of the window a sampling instant?  Every dW-th step from
        the first sampled step s0 on (s0 = 0 for the plain window of Eq. 42,
        s0 = T - |W| for the full-time run of Sec. 4.2.3)."""
        s0, dW = int(self.case.sample_from), int(self.case.sample_every)
        return k >= s0 and (k - s0) % dW == 0

    def sample_weight(self):
        """dW over the sampled span (Eq. 42): 1 / number of samples."""
        return int(self.case.sample_every) / (int(self.case.window_len) - int(self.case.sample_from))

    def run_until_converged(self, p_start=None, gamma=None, max_windows=None):
        """Consecutive windows until Eq. 26 holds (Alg. 1); returns the record."""
        p = self.initial_state() if p_start is None else p_start
        mw = int(max_windows or self.case.max_windows)
        prev = None
        rec = []
        for i in range(mw):
            p_in = p
            p, J, M, _ = self.run_window(p, gamma, store=False)
            ratio, conv = criterion(M, prev, self.case.conv_tol) if prev is not None else (np.inf, False)
            rec.append(dict(window=i, J=J, M=M, ratio=ratio, converged=conv, p_start=p_in, p_end=p))
            prev = M
            if conv:
                break
        return rec

    # -- adjoint -------------------------------------------------------------
    def local_jacobian(self, f, h, aux, g):
        """dp_b / df_a at every node, literally from Eqs. 30-34; shape (Q, Q, N)
        indexed [b, a, node]."""
        lat = self.lat
        c, w, d = lat.c, lat.w, lat.d
        rho, u, pi, pn, te, hneq = (aux[k] for k in ("rho", "u", "pi", "pinorm", "tau_eff", "hneq"))
        cu = c @ u                                               # (Q, N) c_b . u
        uu = (u * u).sum(axis=0)
        cc = c @ c.T                                             # (Q, Q) c_b . c_a
        # Eq. 31: d f^eq_b / d f_a
        first = w[:, None] * (1.0 + cu / CS2 + cu * cu / (2 * CS4) - uu / (2 * CS2))   # (Q, N)
        cb_minus_u_dot_ca_minus_u = cc[:, :, None] - cu[:, None, :] - cu[None, :, :] + uu[None, None]
        cb_dot_ca_minus_u = cc[:, :, None] - cu[:, None, :]
        dfeq = first[:, None, :] + w[:, None, None] * (
            cb_minus_u_dot_ca_minus_u / CS2 + cu[:, None, :] * cb_dot_ca_minus_u / CS4)
        # Eq. 33: d Pi_pq / d f_a
        dpi = -np.einsum("bp,bq,ban->pqan", c, c, dfeq) + np.einsum("ap,aq->pqa", c, c)[..., None]
        # d|Pi|/df_a = 2 Pi:dPi / |Pi|, taken as 0 where |Pi| = 0.
        safe = np.where(pn == 0, 1.0, pn)
        dnorm = np.where(pn == 0, 0.0, 2.0 * np.einsum("pqn,pqan->an", pi, dpi) / safe)
        # Eq. 32: d tau_eff / d f_a
        s = np.sqrt(self.tau ** 2 + 2.0 * self.cs ** 2 * pn / (rho * CS4))
        dtau = self.cs ** 2 / (2.0 * CS4 * s) * (-pn / rho ** 2 + dnorm / rho)     # (Q, N)
        # Eq. 34: d f^neq_b / d f_a (the regularized non-equilibrium part)
        dhneq = w[:, None, None] / (2 * CS4) * np.einsum("bpq,pqan->ban", lat.Qt, dpi)
        om = 1.0 - 1.0 / te
        dh = dfeq + om * dhneq + hneq[:, None, :] * dtau[None] / (te * te)
        # Eq. 30: the partial bounce-back adds g (d h_bbar - d h_b)
        return dh + g[None, None] * (dh[lat.opp] - dh), dict(dh=dh, dpi=dpi, dtau=dtau)

    def objective_source(self, f, h, aux, g, phi, jac_aux):
        """d j / d f_a at every node (the source of Eq. 35) and the direct
        d j / d phi of the objective, both before the sampling weight."""
        lat, case = self.lat, self.case
        k = int(case.obj_kind)
        wv = self.w_obj
        rho, u, pi, te = aux["rho"], aux["u"], aux["pi"], aux["tau_eff"]
        dpi, dtau, dh = jac_aux["dpi"], jac_aux["dtau"], jac_aux["dh"]
        dphi = np.zeros(self.n, dtype=np.result_type(f, g))
        if k == OBJ_DISSIPATION:
            pp = (pi * pi).sum(axis=(0, 1))
            dpp = 2.0 * np.einsum("pqn,pqan->an", pi, dpi)
            # psi = (te - 1/2) pp / (2 rho cs^2 te^2)
            num = (te - 0.5) * pp
            den = 2.0 * rho * CS2 * te * te
            dnum = dtau * pp + (te - 0.5) * dpp
            dden = 2.0 * CS2 * (te * te + rho * 2.0 * te * dtau)
            src = (dnum * den - num * dden) / (den * den)
        elif k == OBJ_VELOCITY_DEV:
            du = u - np.asarray(case.obj_uref, np.float64)[: lat.d, None]
            # d u_p / d f_a = (c_ap - u_p) / rho
            src = 2.0 * np.einsum("pn,apn->an", du, (lat.c[:, :, None] - u[None]) / rho)
        elif k == OBJ_PRESSURE:
            src = np.full((lat.q, self.n), CS2, dtype=f.dtype)
        elif k == OBJ_DRAG:
            cx = lat.c[:, 0]
            src = np.einsum("b,ban->an", cx, g[None, None] * (dh[lat.opp] - dh))
            dg = dg_dphi(phi, case.q_interp, case.g_max)
            dphi = dg * (cx @ (h[lat.opp] - h))
        else:
            raise ValueError("objective kind")
        return wv[None] * src, wv * dphi

    def adjoint_window(self, traj, gamma=None):
        """Backward sweep over one window (Alg. 2 reverse loop, Eqs. 35-36).

        traj holds p^{n0-1} ... p^{n0+|W|-1}.  Returns dJ/dphi per node (Eq. 40
        with the paper's lambda = -a), dJ/dgamma = -dJ/dphi, and a = dJ/dp^{n0-1}.
        """
        lat, case = self.lat, self.case
        W = int(case.window_len)
        weight = self.sample_weight()
        g = self.g(gamma)
        phi = self.phi(gamma)
        dg = dg_dphi(phi, case.q_interp, case.g_max)
        a = np.zeros((lat.q, self.n), dtype=np.result_type(traj[0], g))   # dJ/dp^{n0+W-1}
        grad_phi = np.zeros(self.n, dtype=a.dtype)
        for k in range(W - 1, -1, -1):
            f = self.stream(traj[k])
            h, aux = collide(lat, f, self.tau, self.cs)
            # Eq. 40: d p_b / d phi = g'(phi) (h_bbar - h_b)
            grad_phi += dg * (a * (h[lat.opp] - h)).sum(axis=0)
            jac, jaux = self.local_jacobian(f, h, aux, g)
            b = np.einsum("ban,bn->an", jac, a)                  # Eq. 35
            if self.sampled(k):
                src, dphi = self.objective_source(f, h, aux, g, phi, jaux)
                b = b + weight * src
                grad_phi += weight * dphi
            a = self.stream_adjoint(b)                           # Eq. 36
        return grad_phi, -grad_phi, a

    # -- scalar objective for derivative checks ------------------------------
    def window_objective(self, p_start, gamma):
        """J of one window from a fixed start field, as a function of gamma."""
        _, J, _, _ = self.run_window(p_start, gamma, store=False)
        return J


def criterion(m_cur, m_prev, tol):
    """Consecutive-window test |(M_i - M_{i-1}) / M_i| < eps (Eq. 26).

    Where |M_i| < 1e-30 the absolute difference is used instead.
    """
    diff = abs(m_cur - m_prev)
    ratio = diff if abs(m_cur) < 1e-30 else diff / abs(m_cur)
    return float(ratio), bool(ratio < tol)


def moments_of(lat, p):
    """rho and u of a population field (for comparisons)."""
    rho = density(p)
    return rho, velocity(lat, p, rho)


# ---------------------------------------------------------------------------
# Design pre-processing (Sec. 3.3): density filter of radius r and Heaviside
# projection with threshold eta and steepness beta, and their chain rule.
# ---------------------------------------------------------------------------

def filter_weights(shape, box, radius):
    """Dense matrix of the linear density filter over the design box.

    Inside the box, x~_i = sum_j w_ij x_j / sum_j w_ij with
    w_ij = max(0, r - |x_i - x_j|) over box nodes j; outside the box x~ = x.
    Returned as a scipy sparse matrix acting on the flattened field.
    """
    nz, ny, nx = shape
    x0, x1, y0, y1, z0, z1 = box
    n = nx * ny * nz
    rows, cols, vals = [], [], []
    R = int(np.ceil(radius))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                inside = x0 <= x < x1 and y0 <= y < y1 and z0 <= z < z1
                if not inside:
                    rows.append(i); cols.append(i); vals.append(1.0)
                    continue
                ws, js = [], []
                for dz in range(-R, R + 1):
                    for dy in range(-R, R + 1):
                        for dx in range(-R, R + 1):
                            X, Y, Z = x + dx, y + dy, z + dz
                            if not (x0 <= X < x1 and y0 <= Y < y1 and z0 <= Z < z1):
                                continue
                            w = radius - np.sqrt(dx * dx + dy * dy + dz * dz)
                            if w > 0:
                                ws.append(w)
                                js.append(X + nx * (Y + ny * Z))
                tot = sum(ws)
                rows += [i] * len(js)
                cols += js
                vals += [w / tot for w in ws]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def heaviside(xf, beta, eta):
    """Projection of Wang et al. (2011):
    (tanh(beta eta) + tanh(beta (x - eta))) / (tanh(beta eta) + tanh(beta (1 - eta)))."""
    return (np.tanh(beta * eta) + np.tanh(beta * (xf - eta))) / (np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta)))


def heaviside_derivative(xf, beta, eta):
    return beta * (1.0 - np.tanh(beta * (xf - eta)) ** 2) / (np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta)))


def filter_project(x, shape, box, radius, beta, eta):
    """Raw design x -> filtered -> projected physical field (projection inside the box only)."""
    F = filter_weights(shape, box, radius)
    xf = F @ np.asarray(x).reshape(-1)
    inside = _box_mask(shape, box)
    out = np.where(inside, heaviside(xf, beta, eta), xf)
    return out


def filter_project_adjoint(x, dj_dphys, shape, box, radius, beta, eta):
    """Chain rule: dJ/dx = F^T (H'(x~) * dJ/dphys) (H' = 1 outside the box)."""
    F = filter_weights(shape, box, radius)
    xf = F @ np.asarray(x).reshape(-1)
    inside = _box_mask(shape, box)
    d = np.where(inside, heaviside_derivative(xf, beta, eta), 1.0)
    return F.T @ (d * np.asarray(dj_dphys).reshape(-1))


def _box_mask(shape, box):
    nz, ny, nx = shape
    x0, x1, y0, y1, z0, z1 = box
    m = np.zeros(shape, bool)
    m[z0:z1, y0:y1, x0:x1] = True
    return m.reshape(-1)
