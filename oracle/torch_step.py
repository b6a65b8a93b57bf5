"""Independent plain-PyTorch FP64 statement of one time step (test infrastructure).

This module is part of the oracle: only tests, the smoke check and the CPU
baseline of the benchmark use it.  It restates the same step as the C oracle
(lbm_oracle.c) from the paper, written separately with dense matrices and
precomputed index maps, so that

  * it can be compared with the C oracle on small lattices (two independent
    writings of the same equations), and
  * torch.autograd through it gives FP64 reference gradients of a loss at step
    n with respect to the initial temperature field and the per-node face
    temperatures (the discrete adjoint the CUDA library implements by hand).

Scope: periodic, open (constant-pressure, Sec. 3.3) and bounce-back wall faces
with contact angle 90 degrees (mirror ghost layer of Eq. 36), Peng-Robinson or
ideal-gas EOS, m^eq = M-hat f^eq (or the rows 16-18 printed in Eq. 9).

Step order (one step t -> t+1, every cell):
  1. rho = sum f, j = sum c f, T = sum g; p_EOS and (dp/dT)_rho (Eq. 37); psi (Eq. 7)
  2. F = -G psi(x) sum_i varpi_i psi~(x+c_i) c_i (Eq. 6); u = (j + F/2)/rho (Eq. 5), 0 at walls
  3. D3Q19 MRT collision with the exact-difference forcing (Eq. 8), push streaming
     with bounce-back at walls (Sec. 3.1)
  4. open faces: the general-face form of the Zou-He rules of Sec. 3.3; edge and
     corner nodes of open faces take f^eq(rho_b, 0) for every unknown
  5. D3Q7 collision with the source -w_i Fbar, Fbar = rho c_v u.grad T + T (dp/dT) div u
     (Eqs. 13-15, 27-29), div u by the isotropic D3Q19 difference
  6. relaxed streaming of Eq. 13 with rho c_v at the destination
  7. non-equilibrium extrapolation of g at every node of a non-periodic face (Sec. 3.1)
"""
from __future__ import annotations

import numpy as np
import torch

PERIODIC, WALL, OPEN = 0, 1, 2

# D3Q19 velocities in the order of rows 1-3 of the appendix matrix M-hat
C19 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
                [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=np.int64)
C7 = C19[:7]
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
VARPI = np.array([0.0] + [1 / 6] * 6 + [1 / 12] * 12)  # varpi(|c|^2) of Eq. 6
OPP19 = np.array([0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17])


def mhat_rows(c):
    """Rows of M-hat: the raw moments 1, c, |c|^2, the traceless second moments, the
    third-order c_a^2 c_b and the fourth-order c_a^2 c_b^2 (appendix)."""
    x, y, z = c[:, 0].astype(float), c[:, 1].astype(float), c[:, 2].astype(float)
    return np.stack([np.ones_like(x), x, y, z, x * x + y * y + z * z, 2 * x * x - y * y - z * z, y * y - z * z,
                     x * y, x * z, y * z, x * x * y, x * y * y, x * x * z, x * z * z, y * y * z, y * z * z,
                     x * x * y * y, x * x * z * z, y * y * z * z])


def m7_rows(c):
    """Rows of the D3Q7 matrix M: 1, c_x, c_y, c_z, |c|^2, c_x^2 - c_y^2, c_x^2 - c_z^2 (appendix)."""
    x, y, z = c[:, 0].astype(float), c[:, 1].astype(float), c[:, 2].astype(float)
    return np.stack([np.ones_like(x), x, y, z, x * x + y * y + z * z, x * x - y * y, x * x - z * z])


class TorchStep:
    """The step for one parameter set (a dict with the keys of lbm_params)."""

    def __init__(self, p: dict):
        self.p = dict(p)
        self.n = (int(p["nx"]), int(p["ny"]), int(p["nz"]))
        nx, ny, nz = self.n
        self.N = nx * ny * nz
        self.kind = list(p["face_kind"])
        for fc, k in enumerate(self.kind):
            if k == WALL and float(p["face_theta_deg"][fc]) != 90.0:
                raise NotImplementedError("wetting ghost layer with theta != 90 degrees")
            if k == PERIODIC and int(p.get("face_T_fixed", [0] * 6)[fc]):
                raise NotImplementedError("held temperature layer on a periodic face")
        dt = torch.float64
        self.M = torch.tensor(mhat_rows(C19), dtype=dt)
        self.Minv = torch.linalg.inv(self.M)
        self.M7 = torch.tensor(m7_rows(C7), dtype=dt)
        self.M7inv = torch.linalg.inv(self.M7)
        self.c = torch.tensor(C19, dtype=dt)
        self.w = torch.tensor(W19, dtype=dt)
        self.varpi = torch.tensor(VARPI, dtype=dt)
        wb = float(p["wbar"])
        self.w7 = torch.tensor([1 - wb] + [wb / 6] * 6, dtype=dt)
        self.cs2_7 = wb / 3.0
        self._maps()

    # ------------------------------------------------------------ index maps --
    def _maps(self):
        nx, ny, nz = self.n
        N = self.N
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        X = np.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], 1)  # (N, 3)
        dims = np.array(self.n)
        flat = lambda q: q[:, 0] + nx * (q[:, 1] + ny * q[:, 2])
        # faces of each node (bit fc: on non-periodic face fc)
        m = np.zeros(N, dtype=np.int64)
        for fc in range(6):
            if self.kind[fc] == PERIODIC:
                continue
            a, hi = fc // 2, fc % 2
            m |= ((X[:, a] == (dims[a] - 1 if hi else 0)).astype(np.int64)) << fc
        self.faces = m
        wallbits = sum(1 << fc for fc in range(6) if self.kind[fc] == WALL)
        self.wall_node = torch.tensor((m & wallbits) != 0)

        def ghost(q, rule):
            """Per-axis map of a possibly out-of-range point; rule(kind) for non-periodic faces.
            Returns the mapped flat index and a validity mask (False: zero contribution)."""
            q = q.copy()
            ok = np.ones(len(q), dtype=bool)
            for a in range(3):
                lo, hi = q[:, a] < 0, q[:, a] >= dims[a]
                for side, sel in ((0, lo), (1, hi)):
                    k = self.kind[2 * a + side]
                    if k == PERIODIC:
                        q[sel, a] = np.mod(q[sel, a], dims[a])
                    elif rule == "psi":  # open: copy the boundary node; wall (90 deg): mirror
                        q[sel, a] = (0 if side == 0 else dims[a] - 1) if k == OPEN else \
                            (-q[sel, a] if side == 0 else 2 * (dims[a] - 1) - q[sel, a])
                    else:  # "u": open copy, wall zero
                        if k == OPEN:
                            q[sel, a] = 0 if side == 0 else dims[a] - 1
                        else:
                            ok[sel] = False
                            q[sel, a] = np.clip(q[sel, a], 0, dims[a] - 1)
            return flat(q), ok

        self.psi_src = np.stack([ghost(X + C19[i], "psi")[0] for i in range(19)])  # (19, N)
        us = [ghost(X + C19[i], "u") for i in range(19)]
        self.u_src = np.stack([u[0] for u in us])
        self.u_ok = torch.tensor(np.stack([u[1] for u in us]), dtype=torch.float64)

        # D3Q19 push with bounce-back, as a pull map: slot (i, c) <- slot src19[i, c] of f*
        src = -np.ones(19 * N, dtype=np.int64)
        for i in range(19):
            q = X + C19[i]
            bounce = np.zeros(N, dtype=bool)
            drop = np.zeros(N, dtype=bool)
            for a in range(3):
                for side, sel in ((0, q[:, a] < 0), (1, q[:, a] >= dims[a])):
                    k = self.kind[2 * a + side]
                    if k == PERIODIC:
                        q[sel, a] = np.mod(q[sel, a], dims[a])
                    elif k == WALL:
                        bounce |= sel
                    else:
                        drop |= sel
            cidx = np.arange(N)
            norm = ~bounce & ~drop
            src[i * N + flat(q[norm])] = i * N + cidx[norm]
            src[OPP19[i] * N + cidx[bounce]] = i * N + cidx[bounce]
        self.src19 = src
        # D3Q7 relaxed streaming: source cell of (i, y), -1 beyond a non-periodic face
        s7 = -np.ones((7, N), dtype=np.int64)
        for i in range(7):
            q = X - C7[i]
            ok = np.ones(N, dtype=bool)
            for a in range(3):
                for side, sel in ((0, q[:, a] < 0), (1, q[:, a] >= dims[a])):
                    if self.kind[2 * a + side] == PERIODIC:
                        q[sel, a] = np.mod(q[sel, a], dims[a])
                    else:
                        ok &= ~sel
            s7[i, ok] = flat(q[ok])
        self.src7 = s7
        # open-face nodes: unknown directions, single-face nodes and edges/corners
        self.open_single = {}  # face -> node indices
        self.open_multi = []   # (node, unknown mask, rho_b)
        for c in np.nonzero(m)[0]:
            fcs = [fc for fc in range(6) if (m[c] >> fc) & 1]
            opens = [fc for fc in fcs if self.kind[fc] == OPEN]
            if not opens:
                continue
            if len(fcs) == 1:
                self.open_single.setdefault(opens[0], []).append(c)
            else:
                unk = np.zeros(19, dtype=bool)
                for i in range(1, 19):
                    s = X[c] - C19[i]
                    for a in range(3):
                        if (s[a] < 0 or s[a] >= dims[a]) and self.kind[2 * a] != PERIODIC:
                            unk[i] = True
                rb = np.mean([float(self.p["face_rho"][fc]) for fc in opens])
                self.open_multi.append((c, unk, rb))
        # extrapolation: node, inward node x_f, faces it lies on
        self.nee = []
        for c in np.nonzero(m)[0]:
            q = X[c].copy()
            fcs = [fc for fc in range(6) if (m[c] >> fc) & 1]
            for fc in fcs:
                q[fc // 2] += -1 if fc % 2 else 1
            self.nee.append((c, int(flat(q[None])[0]), fcs, X[c]))

    def face_shape(self, fc):
        a = fc // 2
        t = [b for b in range(3) if b != a]
        return self.n[t[0]], self.n[t[1]]

    def face_index(self, fc, xyz):
        """Index of node xyz in the face array of face fc (lower tangential axis fastest)."""
        a = fc // 2
        t = [b for b in range(3) if b != a]
        return int(xyz[t[0]] + self.n[t[0]] * xyz[t[1]])

    # ---------------------------------------------------------------- physics --
    def eos(self, rho, T):
        """p_EOS and (dp/dT)_rho of Eq. 37 (or the ideal gas p = c0 rho)."""
        p = self.p
        if int(p.get("eos_kind", 0)) == 1:
            return p["eos_c0"] * rho, torch.zeros_like(rho)
        a, b, R, om = p["a"], p["b"], p["R"], p["omega"]
        Tc = 0.0778 * a / (0.45724 * b * R)
        kap = 0.37464 + 1.54226 * om - 0.26992 * om * om
        s = 1.0 + kap * (1.0 - torch.sqrt(T / Tc))
        xi = s * s
        dxi = -kap * s / torch.sqrt(T * Tc)
        den = 1.0 + 2.0 * b * rho - b * b * rho * rho
        pe = rho * R * T / (1.0 - b * rho) - a * xi * rho * rho / den
        dpdT = rho * R / (1.0 - b * rho) - a * dxi * rho * rho / den
        return pe, dpdT

    def feq(self, rho, u):
        cu = self.c @ u  # (19, N)
        uu = (u * u).sum(0)
        return self.w[:, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)

    def meq(self, rho, u):
        me = self.M @ self.feq(rho, u)
        if int(self.p.get("meq_printed", 0)):
            base = rho / 9.0 * (1 - 1.5 * (u * u).sum(0))
            rows = [base + rho / 3 * (u[0] ** 2 + u[1] ** 2), base + rho / 3 * (u[0] ** 2 + u[2] ** 2),
                    base + rho / 3 * (u[1] ** 2 + u[2] ** 2)]
            me = torch.cat([me[:16], torch.stack(rows)], 0)
        return me

    def step(self, f, g, Tface: dict):
        """(f, g) at t -> t+1; f (19, N), g (7, N) FP64 tensors; Tface {face: tensor of face_shape}."""
        p = self.p
        N = self.N
        rho = f.sum(0)
        j = self.c.T @ f  # (3, N)
        T = g.sum(0)
        pe, dpdT = self.eos(rho, T)
        psi = torch.sqrt(2.0 * (pe - rho / 3.0) / p["G"])
        psin = psi[torch.as_tensor(self.psi_src)]  # (19, N)
        S = self.c.T @ (self.varpi[:, None] * psin)  # (3, N)
        F = -p["G"] * psi * S
        notwall = (~self.wall_node).to(f.dtype)
        u = notwall * (j + 0.5 * F) / rho
        ueq = j / rho
        if int(p.get("wall_ueq_zero", 1)):
            ueq = ueq * notwall
        # D3Q19 collision (Eq. 8)
        lam = torch.tensor([1, 1, 1, 1, p["s_e"]] + [p["s_v"]] * 5 + [p["s_q"]] * 6 + [p["s_pi"]] * 3,
                           dtype=f.dtype)[:, None]
        m = self.M @ f
        me0 = self.meq(rho, ueq)
        me1 = self.meq(rho, ueq + F / rho)
        fs = self.Minv @ (m - lam * (m - me0) + me1 - me0)
        # streaming (pull map), then the open faces
        fsf = fs.reshape(-1)
        src = torch.as_tensor(self.src19)
        fo = torch.where(src >= 0, fsf[src.clamp(min=0)], torch.zeros((), dtype=f.dtype)).reshape(19, N).clone()
        for fc, nodes in self.open_single.items():
            fo = self._zouhe(fo, fc, torch.as_tensor(nodes), F, float(p["face_rho"][fc]))
        for c, unk, rb in self.open_multi:
            for i in np.nonzero(unk)[0]:
                fo[i, c] = W19[i] * rb
        # D3Q7 collision with the source
        un = u[:, torch.as_tensor(self.u_src)] * self.u_ok  # (3, 19, N)
        divu = 3.0 * (self.w[:, None] * (self.c.T[:, :, None] * un).sum(0)).sum(0)
        lv, ll = p["lambda_v"], p["lambda_l"]
        if ll == lv:
            lamT = torch.full_like(rho, lv)
        else:
            phi = torch.clamp((rho - p["rho_v"]) / (p["rho_l"] - p["rho_v"]), 0.0, 1.0)
            lamT = lv + (ll - lv) * phi
        vs = 1.0 / (lamT / self.cs2_7 + 0.5)
        mg = self.M7 @ g
        gradT = -vs * mg[1:4] / self.cs2_7
        Fbar = rho * p["cv"] * (u * gradT).sum(0) + T * dpdT * divu
        meq7 = torch.stack([T, 0 * T, 0 * T, 0 * T, p["wbar"] * T, 0 * T, 0 * T])
        lam7 = torch.stack([torch.ones_like(vs), vs, vs, vs, torch.ones_like(vs), torch.ones_like(vs),
                            torch.ones_like(vs)])
        gs = self.M7inv @ (mg - lam7 * (mg - meq7)) - self.w7[:, None] * Fbar
        # relaxed streaming, rho c_v at the destination
        s7 = torch.as_tensor(self.src7)
        gsrc = torch.gather(gs, 1, s7.clamp(min=0))
        go = torch.where(s7 >= 0, g + (gsrc - g) / (rho * p["cv"]), g).clone()
        # extrapolation at every node of a non-periodic face
        rows = []
        for c, cf, fcs, xyz in self.nee:
            Tb = sum(self._face_T(Tface, fc)[self.face_index(fc, xyz)] for fc in fcs) / len(fcs)
            rows.append((c, self.w7 * Tb + go[:, cf] - self.w7 * go[:, cf].sum()))
        if rows:
            go = go.clone()
            idx = torch.as_tensor([r[0] for r in rows])
            go[:, idx] = torch.stack([r[1] for r in rows], 1)
        return fo, go

    def _face_T(self, Tface, fc):
        if Tface is not None and fc in Tface:
            return Tface[fc].reshape(-1)
        return torch.full((int(np.prod(self.face_shape(fc))),), float(self.p["face_T"][fc]), dtype=torch.float64)

    def _zouhe(self, fo, fc, nodes, F, rb):
        """Constant-pressure rule of Sec. 3.3 for face fc (outward normal n), nodes on that face only."""
        a, sg = fc // 2, (1 if fc % 2 else -1)
        cn = sg * C19[:, a]
        Z, P, U = np.nonzero(cn == 0)[0], np.nonzero(cn == 1)[0], np.nonzero(cn == -1)[0]
        fl = fo[:, nodes]
        Fn = sg * F[a, nodes]
        un = (fl[Z].sum(0) + 2 * fl[P].sum(0) + 0.5 * Fn) / rb - 1.0
        fo = fo.clone()
        for i in U:
            t = C19[i].copy()
            t[a] = 0
            if not t.any():
                fo[i, nodes] = fl[OPP19[i]] - rb * un / 3.0
            else:
                corr = 0.0
                for b in range(3):
                    if t[b]:
                        Sb = (torch.tensor(C19[Z, b], dtype=fl.dtype)[:, None] * fl[Z]).sum(0)
                        corr = corr + t[b] * 0.5 * (Sb + 0.5 * F[b, nodes])
                fo[i, nodes] = fl[OPP19[i]] - rb * un / 6.0 - corr + Fn / 8.0
        return fo

    def init_state(self, rho0, T0):
        """f = f^eq(rho0, 0), g = w_i T0 (Sec. 4.2)."""
        u0 = torch.zeros((3, self.N), dtype=torch.float64)
        return self.feq(rho0, u0), self.w7[:, None] * T0
