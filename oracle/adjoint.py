"""FP64 CPU discrete adjoint of the coupled 2-D step (test infrastructure).

Only the tests and the gradient leg of ``bench.py`` import this module; the
CUDA library and its binding never do.

What it computes.  The gradient, with respect to theta = (ln A, Ta, T_wall,
u_in), of an objective of the state after n steps: the flame position
J = dx * sum_fluid Y_F / (Y_F,in * fluid cells of the x = 0 section)
(Sec. IV.A: the flame is located from the unburnt fuel), or the quenching
distance J = (sum h d^-4 / sum h)^(-1/4) (a heat-release-weighted soft
minimum of the distance d from a cell to the nearest cold wall, standing in
for the dead-zone thickness of Sec. IV.A), as the transpose of the
derivative of the discrete D2Q9 step, lambda^n = (dF/dx^n)^T lambda^{n+1},
accumulated in reverse over the steps.

How.  The step is restated here with plain PyTorch CPU operations in FP64,
vectorised over the fluid cells, in the order of the oracle (``orc.c``):
a1 pull-streaming with half-way bounce-back (Eq. 28), the Eq. 31 inlet, the
Eq. 32 convective outlet and the constant-pressure outlet; a2 EOS density
and the first moment (Eq. 13b); a3 ghost points per axis line (Eq. 34 on a
staircase mask: Dirichlet 2 phi_B - phi_I, Neumann phi_I); a4 WENO3 or
centred convection with the species correction (Eq. 26); a5 4th-order
diffusion with the mixture-averaged flux (Eq. 1, 2, 7); a6 the single-step
Arrhenius rate; a7 explicit Euler and Lambda (Eq. 6); a8-a9 Xi, P_h,
pre-conditioning and the cumulant collision (Eq. 9, 13a, 19, 21-23) with the
central-moment matrix inverted by a linear solve.  The readings are those of
the oracle (its header lists them).  Reverse accumulation is
``torch.autograd`` (a library primitive); ``checkpoint_every`` recomputes
each segment of steps in the backward sweep instead of keeping its tape.

Branch decisions (WENO upwind side on the sign of u, max(Y, 0) in the rate,
the geometry's near-boundary switches) are taken on the values, so the
result is the derivative of the discrete map where it is differentiable.

Pins (``tests/test_oracle_adjoint.py``): the forward step equals the C
oracle's step to rounding on every boundary type; the gradient equals
central differences of the C oracle's J.
"""
from __future__ import annotations

import math

import numpy as np
import torch

CS2 = 1.0 / 3.0
CS = math.sqrt(CS2)
# D2Q9, population i = (cx + 1) + 3 (cy + 1); weights are products of the
# D1Q3 weights {1/6, 2/3, 1/6}
_C = [(i % 3 - 1, i // 3 - 1) for i in range(9)]
_W1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
_WGT = [_W1[cx] * _W1[cy] for cx, cy in _C]
_OPP = [(-cx + 1) + 3 * (-cy + 1) for cx, cy in _C]

# kinds of a pulled population
STREAM, BOUNCE, INLET, OUTLET_P, OUTLET_C = range(5)
# kinds of an FD line point
P_FLUID, P_NEUMANN, P_DIRICHLET_T, P_INLET = range(4)
# boundary types (as in the oracle's configuration)
PERIODIC, WALL_AD, WALL_ISO, BC_INLET, BC_OUTLET, BC_OUTLET_P = range(6)
_BC = {"periodic": 0, "wall_adiabatic": 1, "wall_isothermal": 2, "inlet": 3, "outlet": 4, "outlet_pressure": 5}
_SOLID = -1


class Geometry:
    """Per fluid cell tables of the pull rules and of the FD line points,
    built once from the mask and the face types by the rules of Sec. III
    (plain Python loops over the cells)."""

    def __init__(self, cfg: dict, solid: np.ndarray):
        self.solid_iso = bool(cfg["solid_isothermal"])
        if cfg["dim"] != 2:
            raise ValueError("the CPU adjoint restates the 2-D (D2Q9) step")
        self.nx, self.ny = cfg["nx"], cfg["ny"]
        self.bc = [_BC[b] for b in cfg["bc"]]
        self.solid = np.asarray(solid, dtype=np.uint8).reshape(self.ny, self.nx)
        nx, ny = self.nx, self.ny
        self.fluid = np.array([x + nx * y for y in range(ny) for x in range(nx) if not self.solid[y, x]],
                              dtype=np.int64)
        F = self.fluid.size
        # pull tables [9][F]
        self.pkind = np.zeros((9, F), np.int64)
        self.psrc = np.zeros((9, F), np.int64)    # STREAM source, OUTLET_C inner cell
        self.pface = np.zeros((9, F), np.int64)   # inlet / outlet face
        for f, c in enumerate(self.fluid):
            x, y = c % nx, c // nx
            for i, (cx, cy) in enumerate(_C):
                k, s, face = self._pull_rule(x, y, cx, cy)
                self.pkind[i, f], self.psrc[i, f], self.pface[i, f] = k, s, face
        # FD line tables [axis][5][F]: kind, source cell, Dirichlet face (or -1 for a solid)
        self.lkind = np.zeros((2, 5, F), np.int64)
        self.lsrc = np.zeros((2, 5, F), np.int64)
        self.lface = np.full((2, 5, F), -2, np.int64)
        self.near = np.zeros((2, F), bool)
        for f, c in enumerate(self.fluid):
            x, y = c % nx, c // nx
            for a in range(2):
                near, pts = self._line(x, y, a)
                self.near[a, f] = near
                for j, (k, s, face) in enumerate(pts):
                    self.lkind[a, j, f], self.lsrc[a, j, f], self.lface[a, j, f] = k, s, face
        self.section = int(sum(1 for y in range(ny) if not self.solid[y, 0]))
        self.wall_distance = np.array([self._wall_distance(c % nx, c // nx) for c in self.fluid])
        self.inlet_y = np.array([c // nx for c in self.fluid], dtype=np.float64) + 0.5

    # --- classification of a lattice position (periodic axes wrapped) ----
    def _classify(self, x, y):
        p = [x, y]
        n = [self.nx, self.ny]
        face = -1
        for a in range(2):
            f = -1
            if p[a] < 0:
                f = 2 * a
            elif p[a] >= n[a]:
                f = 2 * a + 1
            if f < 0:
                continue
            if self.bc[f] == PERIODIC:
                p[a] %= n[a]
            elif face < 0:
                face = f
        if face >= 0:
            return "face", face
        c = p[0] + self.nx * p[1]
        return ("solid", c) if self.solid[p[1], p[0]] else ("fluid", c)

    def _pull_rule(self, x, y, cx, cy):
        src = [x - cx, y - cy]
        n = [self.nx, self.ny]
        wall, inlet, outlet = False, -1, -1
        for a in range(2):
            f = -1
            if src[a] < 0:
                f = 2 * a
            elif src[a] >= n[a]:
                f = 2 * a + 1
            if f < 0:
                continue
            b = self.bc[f]
            if b == PERIODIC:
                src[a] %= n[a]
            elif b == BC_INLET:
                inlet = f if inlet < 0 else inlet
            elif b in (BC_OUTLET, BC_OUTLET_P):
                outlet = f if outlet < 0 else outlet
            else:
                wall = True
        if not wall and (inlet >= 0 or outlet >= 0):
            q = [min(max(src[a], 0), n[a] - 1) for a in range(2)]
            if self.solid[q[1], q[0]]:
                wall = True  # a link through an inlet/outlet face next to a solid cell hits the solid
        c = x + self.nx * y
        if wall:
            return BOUNCE, c, -1
        if inlet >= 0:
            return INLET, c, inlet
        if outlet >= 0 and self.bc[outlet] == BC_OUTLET_P:
            return OUTLET_P, c, outlet
        if outlet >= 0:
            a, nsign = outlet // 2, (1 if outlet % 2 else -1)
            q = [x, y]
            q[a] -= nsign
            inner = c
            if 0 <= q[a] < n[a] and not self.solid[q[1], q[0]]:
                inner = q[0] + self.nx * q[1]
            return OUTLET_C, inner, outlet
        s = src[0] + self.nx * src[1]
        if self.solid[src[1], src[0]]:
            return BOUNCE, c, -1
        return STREAM, s, -1

    def _wall_distance(self, x, y, cap=64):
        """Distance (cells, to the wall plane half-way between cells) to the
        nearest cold boundary along the four axis directions: an isothermal
        solid cell (when solids are isothermal) or the layer beyond an
        isothermal wall face; periodic faces are crossed; `cap` if none."""
        best = float(cap)
        n = [self.nx, self.ny]
        for a in range(2):
            for side in (-1, 1):
                for j in range(1, cap + 1):
                    if j - 0.5 >= best:
                        break
                    q = [x, y]
                    q[a] += side * j
                    if q[a] < 0 or q[a] >= n[a]:
                        f = 2 * a + (0 if q[a] < 0 else 1)
                        if self.bc[f] == PERIODIC:
                            q[a] %= n[a]
                        else:
                            if self.bc[f] == WALL_ISO:
                                best = j - 0.5
                            break
                    if self.solid[q[1], q[0]]:
                        if self.solid_iso:
                            best = j - 0.5
                        break
        return best

    def _ghost_kind(self, kind, face):
        """(line point kind, Dirichlet face or -1 for a solid) of a ghost
        whose wall is a solid cell (face = None) or a domain face."""
        if face is None:
            return (P_DIRICHLET_T, -1) if self.solid_iso else (P_NEUMANN, -2)
        b = self.bc[face]
        if b == WALL_ISO:
            return P_DIRICHLET_T, face
        if b == BC_INLET:
            return P_INLET, face
        return P_NEUMANN, -2

    def _line(self, x, y, a):
        """The five points (offsets -2..2) of the FD line through (x, y)
        along axis a: (kind, source cell, face).  Ghost rule (Eq. 34 on the
        mask): the ghost at distance j beyond a wall at distance w mirrors
        the point at offset 2w - 1 - j; offset -1 is the fluid neighbour on
        the other side, or the centre when that is not fluid."""
        c = x + self.nx * y
        pts = [None] * 5
        pts[2] = (P_FLUID, c, -2)
        near = False
        for side in (-1, 1):
            w, wk, wf = 0, None, None
            for j in (1, 2):
                q = [x, y]
                q[a] += side * j
                t, v = self._classify(*q)
                if t == "fluid":
                    pts[2 + side * j] = (P_FLUID, v, -2)
                else:
                    w = j
                    wk, wf = t, (v if t == "face" else None)
                    break
            if not w:
                continue
            near = True
            kind, face = self._ghost_kind(wk, wf)
            for j in range(w, 3):
                m = 2 * w - 1 - j
                if m >= 0:
                    src = pts[2 + side * m][1]
                else:
                    q = [x, y]
                    q[a] -= side
                    t, v = self._classify(*q)
                    src = v if t == "fluid" else c
                pts[2 + side * j] = (kind, src, face)
        return near, pts


def _d1(v):
    return (v[0] - 8.0 * v[1] + 8.0 * v[3] - v[4]) / 12.0


def _d2(v):
    return (-v[0] + 16.0 * v[1] - 30.0 * v[2] + 16.0 * v[3] - v[4]) / 12.0


def _c2(v):
    return 0.5 * (v[3] - v[1])


def _weno_face(a, b, c, eps):
    q0 = -0.5 * a + 1.5 * b
    q1 = 0.5 * b + 0.5 * c
    b0 = (b - a) * (b - a)
    b1 = (c - b) * (c - b)
    a0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0))
    a1 = (2.0 / 3.0) / ((eps + b1) * (eps + b1))
    return (a0 * q0 + a1 * q1) / (a0 + a1)


def _weno3(v, u, eps):
    """Jiang-Shu WENO3 derivative at the centre of v[0..4], upwinded on the
    sign of u (u = 0 takes the u >= 0 side)."""
    pos = _weno_face(v[1], v[2], v[3], eps) - _weno_face(v[0], v[1], v[2], eps)
    neg = _weno_face(v[4], v[3], v[2], eps) - _weno_face(v[3], v[2], v[1], eps)
    return torch.where(u >= 0.0, pos, neg)


class Step:
    """The coupled D2Q9 step in FP64 PyTorch, differentiable in the state
    and in theta = (ln A, Ta, T_wall, u_in)."""

    def __init__(self, cfg: dict, solid: np.ndarray):
        self.cfg = dict(cfg)
        self.geo = Geometry(cfg, solid)
        g = self.geo
        t = lambda a: torch.as_tensor(a)
        self.fluid = t(g.fluid)
        self.pkind, self.psrc, self.pface = t(g.pkind), t(g.psrc), t(g.pface)
        self.lkind, self.lsrc, self.lface = t(g.lkind), t(g.lsrc), t(g.lface)
        self.near = t(g.near)
        # base Dirichlet temperatures of the line points (cfg values)
        tb = np.full(g.lkind.shape, float(cfg["T_in"]))  # (unused where not Dirichlet; kept finite)
        Twall = np.asarray(cfg["T_wall"], dtype=np.float64)
        tb = np.where(g.lkind == P_INLET, cfg["T_in"], tb)
        tb = np.where((g.lkind == P_DIRICHLET_T) & (g.lface >= 0), Twall[np.clip(g.lface, 0, 5)], tb)
        tb = np.where((g.lkind == P_DIRICHLET_T) & (g.lface == -1), cfg["T_solid"], tb)
        self.TB0 = t(tb)
        self.Tw0 = float(self.theta0()[2])
        self.N = g.nx * g.ny
        self.W = torch.tensor(cfg["W"], dtype=torch.float64)
        self.Y_in = torch.tensor(cfg["Y_in"], dtype=torch.float64)
        self.invW_in = float((self.Y_in / self.W).sum())
        self.nu_stoich = list(cfg["nu_stoich"])
        self.alpha = cfg["nu"] / cfg["Pr"]
        self.D = [self.alpha / le for le in cfg["Le"]]
        self.omega_s = 1.0 / (cfg["nu"] / CS2 + 0.5)
        self.omega_b = cfg["omega_bulk"] if cfg["omega_bulk"] > 0 else self.omega_s
        self.omega_hi = cfg["omega_hi"]
        # population constants
        self.cx = torch.tensor([c[0] for c in _C], dtype=torch.float64)
        self.cy = torch.tensor([c[1] for c in _C], dtype=torch.float64)
        self.w = torch.tensor(_WGT, dtype=torch.float64)
        self.opp = _OPP
        fuel, ox = cfg["fuel"], cfg["oxidiser"]
        self.fuel, self.ox = fuel, ox
        self.yield_ = [cfg["nu_stoich"][k] * cfg["W"][k] / (-cfg["nu_stoich"][fuel] * cfg["W"][fuel])
                       for k in range(5)]

    def theta0(self):
        cfg = self.cfg
        walls = [cfg["T_wall"][f] for f, b in enumerate(cfg["bc"]) if b == "wall_isothermal"]
        Tw = walls[0] if walls else cfg["T_solid"]
        return torch.tensor([math.log(cfg["A"]), cfg["Ta"], Tw, cfg["u_in"]], dtype=torch.float64)

    def eos(self, T, invW):
        return (self.cfg["T_in"] / T) * (self.invW_in / invW)

    def __call__(self, g, T, Y, theta):
        """One step: (g[9,N], T[N], Y[5,N]) -> the next state.  Solid cells
        keep their values."""
        cfg = self.cfg
        lnA, Ta, Tw, u_in = theta[0], theta[1], theta[2], theta[3]
        fl = self.fluid
        F = fl.numel()
        # Dirichlet temperature of each line point: T_wall of its face or
        # T_solid, all moved together by theta's T_wall (T_in at an inlet)
        dTw = Tw - self.Tw0
        invW_all = (Y / self.W[:, None]).sum(0)
        rho_all = self.eos(T, invW_all)
        # a1: pull-streaming and boundary rules
        gin = []
        rho_c = rho_all[fl]
        # outlets use rho of the stored scalars and u of the stored populations
        ux = (self.cx[:, None] * g[:, fl]).sum(0) / (rho_c * CS2)
        uy = (self.cy[:, None] * g[:, fl]).sum(0) / (rho_c * CS2)
        uu = ux * ux + uy * uy
        for i in range(9):
            k, s, face = self.pkind[i], self.psrc[i], self.pface[i]
            ib = self.opp[i]
            out = g[i, s]  # STREAM (s is the source); OUTLET_C inner
            bounce = g[ib, fl]
            out = torch.where(k == BOUNCE, bounce, out)
            # inlet: u_in along the inward normal, plug or Poiseuille profile
            sgn = torch.where(face % 2 == 0, 1.0, -1.0).to(torch.float64)
            mag = u_in * torch.ones(F, dtype=torch.float64)
            if cfg["poiseuille_inlet"]:
                ny = float(self.geo.ny)
                yy = torch.as_tensor(self.geo.inlet_y)
                mag = torch.where(face // 2 == 0, 6.0 * u_in * yy * (ny - yy) / (ny * ny), mag)
            cvec = torch.where(face // 2 == 0, self.cx[i], self.cy[i])
            inl = bounce + (self.w[i] + self.w[ib]) * 1.0 * cvec * sgn * mag
            out = torch.where(k == INLET, inl, out)
            cu = self.cx[i] * ux + self.cy[i] * uy
            geq_even = self.w[i] * (0.0 - rho_c * CS2) + CS2 * self.w[i] * rho_c * (
                1.0 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2))
            out = torch.where(k == OUTLET_P, -bounce + 2.0 * geq_even, out)
            nsign = torch.where(face % 2 == 1, 1.0, -1.0).to(torch.float64)
            un = torch.where(face // 2 == 0, ux, uy) * nsign
            conv = (CS - un) * g[i, s] + (1.0 - CS + un) * g[i, fl]
            out = torch.where(k == OUTLET_C, conv, out)
            gin.append(out)
        gin = torch.stack(gin)
        # a2: density (EOS) and velocity (Eq. 13b)
        Tc = T[fl]
        Yc = Y[:, fl]
        invWc = invW_all[fl]
        rho = rho_c
        u = [(self.cx[:, None] * gin).sum(0) / (rho * CS2), (self.cy[:, None] * gin).sum(0) / (rho * CS2)]
        # a3-a5: FD lines
        epsY = cfg["weno_eps"]
        epsT = cfg["weno_eps"] * cfg["T_in"] ** 2
        conv_T = torch.zeros(F, dtype=torch.float64)
        diff_T = torch.zeros(F, dtype=torch.float64)
        conv_Y = [torch.zeros(F, dtype=torch.float64) for _ in range(5)]
        diff_Y = [torch.zeros(F, dtype=torch.float64) for _ in range(5)]
        grad_rho = []
        for a in range(2):
            Tl, Yl, rl = [], [], []
            for j in range(5):
                k, s, face = self.lkind[a, j], self.lsrc[a, j], self.lface[a, j]
                Ts, Ys, rs = T[s], Y[:, s], rho_all[s]
                TB = self.TB0[a, j] + torch.where(k == P_INLET, torch.zeros_like(Ts), dTw * torch.ones_like(Ts))
                dirT = (k == P_DIRICHLET_T) | (k == P_INLET)
                Tj = torch.where(dirT, 2.0 * TB - Ts, Ts)
                Yj = torch.where((k == P_INLET)[None, :], 2.0 * self.Y_in[:, None] - Ys, Ys)
                YB = torch.where((k == P_INLET)[None, :], self.Y_in[:, None].expand_as(Ys), Ys)
                rhoB = self.eos(TB, (YB / self.W[:, None]).sum(0))
                rj = torch.where(dirT, 2.0 * rhoB - rs, rs)
                Tl.append(Tj)
                Yl.append(Yj)
                rl.append(rj)
            invWl = [(Yl[j] / self.W[:, None]).sum(0) for j in range(5)]
            Xl = [Yl[j] / (self.W[:, None] * invWl[j][None, :]) for j in range(5)]
            near = self.near[a]
            drho = _d1(rl)
            grad_rho.append(drho)
            ua = u[a]
            conv_T = conv_T + ua * torch.where(near, _c2(Tl), _weno3(Tl, ua, epsT))
            diff_T = diff_T + self.alpha * (_d2(Tl) + drho * _d1(Tl) / rho)
            L = []
            for k in range(5):
                v = [Yl[j][k] for j in range(5)]
                L.append(torch.where(near, _c2(v), _weno3(v, ua, epsY)))
            sumL = L[0] + L[1] + L[2] + L[3] + L[4]
            for k in range(5):
                conv_Y[k] = conv_Y[k] + ua * (L[k] - Yc[k] * sumL)
            dinvW = _d1(invWl)
            m, dm, dY = [], [], []
            for k in range(5):
                ak = self.D[k] * cfg["W"][k]
                v = [Xl[j][k] for j in range(5)]
                dX, d2X = _d1(v), _d2(v)
                m.append(ak * invWc * dX)
                dm.append(ak * (invWc * d2X + dinvW * dX))
                dY.append(_d1([Yl[j][k] for j in range(5)]))
            Msum = m[0] + m[1] + m[2] + m[3] + m[4]
            dMsum = dm[0] + dm[1] + dm[2] + dm[3] + dm[4]
            for k in range(5):
                diff_Y[k] = diff_Y[k] + dm[k] - dY[k] * Msum - Yc[k] * dMsum + (m[k] - Yc[k] * Msum) * drho / rho
        # a6: reaction, q = A dt max(Y_F,0) max(Y_O,0) exp(-Ta/T)
        yf = torch.where(Yc[self.fuel] > 0.0, Yc[self.fuel], torch.zeros_like(Tc))
        yo = torch.where(Yc[self.ox] > 0.0, Yc[self.ox], torch.zeros_like(Tc))
        q = torch.exp(lnA) * cfg["dt"] * yf * yo * torch.exp(-Ta / Tc)
        reac_T = cfg["Q"] / cfg["cp"] * q
        # a7: explicit Euler, Lambda from the non-convective rates (Eq. 6)
        T_new = Tc + (-conv_T + diff_T + reac_T)
        Lam = (diff_T + reac_T) / Tc
        Wmix = 1.0 / invWc
        Y_new = []
        for k in range(5):
            rk = self.yield_[k] * q
            Y_new.append(Yc[k] + (-conv_Y[k] + diff_Y[k] + rk))
            Lam = Lam + Wmix / cfg["W"][k] * (diff_Y[k] + rk)
        # a8-a9: Xi, P_h, pre-conditioning, cumulant collision
        gstar = self.collide(gin, rho, u, grad_rho, Lam)
        g2 = g.index_copy(1, fl, gstar)
        T2 = T.index_copy(0, fl, T_new)
        Y2 = Y.index_copy(1, fl, torch.stack(Y_new))
        return g2, T2, Y2

    def collide(self, gin, rho, u, grad_rho, Lam):
        ux, uy = u
        cx, cy, w = self.cx[:, None], self.cy[:, None], self.w[:, None]
        P_h = gin.sum(0) + 0.5 * rho * CS2 * Lam                          # Eq. 13a
        cu = cx * ux + cy * uy
        uu = ux * ux + uy * uy
        feq = w * rho * (1.0 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2))   # Eq. 10
        cmg = (cx - ux) * grad_rho[0] + (cy - uy) * grad_rho[1]
        Xi = CS2 * (feq / rho - w) * cmg + w * rho * CS2 * Lam           # Eq. 9
        geq = w * (P_h - rho * CS2) + CS2 * feq                            # Eq. 12
        fp = gin / (rho * CS2) + Xi / (2.0 * rho * CS2)                    # Eq. 19
        fpeq = geq / (rho * CS2)
        # central-moment matrix M[j, i] = (c_ix - u_x)^p (c_iy - u_y)^q, j = p + 3q (Eq. 21)
        dx = (self.cx[None, :] - ux[:, None])   # [F, 9]
        dy = (self.cy[None, :] - uy[:, None])
        one = torch.ones_like(dx)
        px = [one, dx, dx * dx]   # explicit powers: pow(0, 0) has no usable derivative
        py = [one, dy, dy * dy]
        rows = []
        for j in range(9):
            rows.append(px[j % 3] * py[j // 3])
        M = torch.stack(rows, dim=1)            # [F, 9 (j), 9 (i)]
        Pi = torch.einsum("fji,if->fj", M, fp)
        Pieq = torch.einsum("fji,if->fj", M, fpeq)
        XX, YY, XY, XXYY = 2, 6, 4, 8

        def cumulants(P):
            K = P.clone()
            K[:, XXYY] = P[:, XXYY] - P[:, XX] * P[:, YY] - 2.0 * P[:, XY] * P[:, XY]   # Eq. 22
            return K

        K, Keq = cumulants(Pi), cumulants(Pieq)
        ws, wb, wh = self.omega_s, self.omega_b, self.omega_hi
        Ks = [None] * 9
        for j in range(9):
            order = j % 3 + j // 3
            if order <= 1:
                Ks[j] = K[:, j]
            elif order >= 3:
                Ks[j] = Keq[:, j] + (1.0 - wh) * (K[:, j] - Keq[:, j])
        tr, treq = K[:, XX] + K[:, YY], Keq[:, XX] + Keq[:, YY]
        dv, dveq = K[:, XX] - K[:, YY], Keq[:, XX] - Keq[:, YY]
        trs = treq + (1.0 - wb) * (tr - treq)
        dvs = dveq + (1.0 - ws) * (dv - dveq)
        Ks[XX] = 0.5 * (trs + dvs)
        Ks[YY] = 0.5 * (trs - dvs)
        Ks[XY] = Keq[:, XY] + (1.0 - ws) * (K[:, XY] - Keq[:, XY])
        Ks = torch.stack(Ks, dim=1)
        Pis = Ks.clone()
        Pis[:, XXYY] = Ks[:, XXYY] + Ks[:, XX] * Ks[:, YY] + 2.0 * Ks[:, XY] * Ks[:, XY]
        fps = torch.linalg.solve(M, Pis.unsqueeze(-1)).squeeze(-1).T       # back to [9, F]
        return rho * CS2 * fps + 0.5 * Xi                                   # Eq. 14

    def flame_position(self, Y):
        """J = dx * sum_fluid Y_F / (Y_F,in * fluid cells of the x = 0 section) [m]."""
        return self.cfg["dx"] * Y[self.fuel, self.fluid].sum() / (self.cfg["Y_in"][self.fuel] * self.geo.section)

    def quench_distance(self, T, Y, theta):
        """J = (sum_fluid h d^-4 / sum_fluid h)^(-1/4) [cells], h = rho (Q/cp) q
        the heat release of a cell (the rate with theta's A and Ta) and d its
        distance to the nearest cold wall."""
        cfg = self.cfg
        fl = self.fluid
        Tc, Yc = T[fl], Y[:, fl]
        rho = self.eos(Tc, (Yc / self.W[:, None]).sum(0))
        yf = torch.where(Yc[self.fuel] > 0.0, Yc[self.fuel], torch.zeros_like(Tc))
        yo = torch.where(Yc[self.ox] > 0.0, Yc[self.ox], torch.zeros_like(Tc))
        h = rho * cfg["Q"] / cfg["cp"] * torch.exp(theta[0]) * cfg["dt"] * yf * yo * torch.exp(-theta[1] / Tc)
        w = torch.as_tensor(self.geo.wall_distance) ** -4.0
        return ((h * w).sum() / h.sum()) ** -0.25

    def objective(self, name, g, T, Y, theta):
        if name == "flame_position":
            return self.flame_position(Y)
        if name == "quench_distance":
            return self.quench_distance(T, Y, theta)
        raise ValueError(name)


def _to_t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64))


def forward(cfg, solid, T0, Y0, g0, steps: int, theta=None):
    """The state after `steps` steps (numpy arrays), no gradient."""
    st = Step(cfg, solid)
    th = st.theta0() if theta is None else torch.as_tensor(theta, dtype=torch.float64)
    g = _to_t(g0).reshape(9, -1).clone()
    T, Y = _to_t(T0).clone(), _to_t(Y0).reshape(5, -1).clone()
    with torch.no_grad():
        for _ in range(steps):
            g, T, Y = st(g, T, Y, th)
    return g.numpy(), T.numpy(), Y.numpy()


def adjoint_gradient(cfg, solid, T0, Y0, steps: int, checkpoint_every: int = 0, g0=None, theta=None,
                     objective: str = "flame_position"):
    """(J, dJ/dtheta) of the objective (flame_position or quench_distance)
    after `steps` steps from (T0, Y0, g0 = 0 by default), by reverse
    accumulation over the steps.
    checkpoint_every > 0 keeps only the state at the start of each segment
    of that many steps and recomputes the segment's tape in the backward
    sweep."""
    from torch.utils.checkpoint import checkpoint

    st = Step(cfg, solid)
    th = (st.theta0() if theta is None else torch.as_tensor(theta, dtype=torch.float64)).clone()
    th.requires_grad_(True)
    N = st.N
    g = torch.zeros(9, N, dtype=torch.float64) if g0 is None else _to_t(g0).reshape(9, N).clone()
    T, Y = _to_t(T0).clone(), _to_t(Y0).reshape(5, -1).clone()

    def segment(n, g, T, Y, th):
        for _ in range(n):
            g, T, Y = st(g, T, Y, th)
        return g, T, Y

    done = 0
    while done < steps:
        n = steps - done if checkpoint_every <= 0 else min(checkpoint_every, steps - done)
        if checkpoint_every > 0:
            g, T, Y = checkpoint(segment, n, g, T, Y, th, use_reentrant=False)
        else:
            g, T, Y = segment(n, g, T, Y, th)
        done += n
    J = st.objective(objective, g, T, Y, th)
    (grad,) = torch.autograd.grad(J, th)
    return float(J.detach()), grad.numpy()
