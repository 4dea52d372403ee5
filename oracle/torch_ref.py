"""TEST INFRASTRUCTURE ONLY: a plain PyTorch (CPU, FP64) composition of the HOPE forward
operator, built from the C oracle's tables, whose torch.autograd gradient is the slow
reference against which the CUDA library's hand-written adjoint is checked.

Every step follows the same equations as the C oracle (arXiv 2411.19185: ghost iteration
of section 3.3.1 with the conversions of eqs. 3.26-3.29, TPP of eqs. 3.14-3.15 or the
WENO-Z combination of eqs. 3.20-3.25, LMARS of eqs. 3.31-3.38 with the single-flux rule
at panel edges, sources of eqs. 2.2-2.3, quadrature of eqs. 3.5-3.6, SSP-RK3), written as
whole-array tensor operations so that autograd can differentiate them.  Its forward is
checked against the C oracle before its gradient is trusted.
"""
import numpy as np
import torch

from . import oracle as O


class TorchReference:
    def __init__(self, N, k, scheme=O.TPP, radius=O.RADIUS, gravity=O.GRAVITY, omega=O.OMEGA,
                 weno_eps=1e-40, ghost_iters=10, coriolis_tilt=0.0):
        o = O.Oracle(N, k, scheme, radius, gravity, omega, weno_eps, ghost_iters, coriolis_tilt)
        self.o, self.N, self.k, self.scheme = o, N, k, scheme
        self.H, self.me, self.ne = o.H, o.me, N + 2 * o.H
        self.r, self.omega, self.eps, self.iters = radius, omega, weno_eps, ghost_iters
        H, me, ne, K = self.H, self.me, self.ne, k
        self.dx = np.pi / (2 * N)
        gx, gw = O.gauss(me)
        self.gx, self.gw = gx, torch.tensor(gw)
        xi, eta = o.points()
        self.npoc = len(xi)
        # TPP weights per point: R[pt, b*K + a]
        self.R = torch.tensor(np.stack([O.tpp_weights_2d(K, xi[p], eta[p]).ravel() for p in range(self.npoc)]))
        # stencils of every interior cell into the flattened extended panel array
        cj, ci = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        bb, aa = np.meshgrid(np.arange(K), np.arange(K), indexing="ij")
        loc = (cj[..., None, None] + bb) * ne + (ci[..., None, None] + aa)  # (N, N, K, K)
        st = np.stack([p * ne * ne + loc for p in range(6)]).reshape(6 * N * N, K * K)
        self.st_idx = torch.tensor(st)
        if scheme == O.WENO:
            l = (k + 1) // 2
            s = l * l
            self.l, self.s = l, s
            rsub = np.zeros((self.npoc, s, l * l))
            gp, gm = np.zeros((self.npoc, s)), np.zeros((self.npoc, s))
            for p in range(self.npoc):
                for sy in range(l):
                    for sx in range(l):
                        rx = O.weights_1d(l, sx - H, xi[p])
                        ry = O.weights_1d(l, sy - H, eta[p])
                        rsub[p, sy * l + sx] = np.outer(ry, rx).ravel()
                g, _ = O.weno_gamma(k, xi[p], eta[p])
                g = g.ravel()
                gp[p] = 0.5 * (3 * np.abs(g) + g)
                gm[p] = 0.5 * (3 * np.abs(g) - g)
            self.rsub = torch.tensor(rsub)
            self.gp, self.gm = torch.tensor(gp), torch.tensor(gm)
            self.sp, self.sm = self.gp.sum(1), self.gm.sum(1)
            # sub-stencil cells inside the K x K stencil, and the indicators as quadratic
            # forms beta = q^T M q, M obtained from the oracle's beta by polarisation
            sub = np.zeros((s, l * l), np.int64)
            M = np.zeros((s, l * l, l * l))
            for sy in range(l):
                for sx in range(l):
                    i = sy * l + sx
                    for b in range(l):
                        for a in range(l):
                            sub[i, b * l + a] = (sy + b) * K + (sx + a)
                    e = np.eye(l * l)
                    d = np.array([O.weno_beta(l, sx - H, sy - H, e[u]) for u in range(l * l)])
                    for u in range(l * l):
                        M[i, u, u] = d[u]
                        for w in range(u + 1, l * l):
                            v = 0.5 * (O.weno_beta(l, sx - H, sy - H, e[u] + e[w]) - d[u] - d[w])
                            M[i, u, w] = M[i, w, u] = v
            self.sub_idx = torch.tensor(sub)
            self.M = torch.tensor(M)
        # ghost Gauss points
        gt = o.ghost_tables()
        ring = gt["ring"]
        nr = len(ring)
        self.ring_idx = torch.tensor(np.concatenate([p * ne * ne + ring for p in range(6)]))
        src = []
        for r in range(len(gt["B"])):
            B, ic, jc = gt["B"][r], gt["ic"][r], gt["jc"][r]
            src.append(B * ne * ne + ((jc + bb) * ne + (ic + aa)).ravel())
        self.g_src = torch.tensor(np.array(src))
        self.g_w = torch.tensor(np.einsum("rb,ra->rba", gt["wy"], gt["wx"]).reshape(-1, K * K))
        self.g_ratio = torch.tensor(gt["ratio"] * gt["w"])  # two owner slots per point, shares w
        self.g_C = torch.tensor(gt["C"] * gt["w"][:, None])
        W = np.outer(gw, gw).ravel()  # [h*me + g]
        self.g_W = torch.tensor(W)
        # metric terms at the edge points: x-edges (X_e, Y_jg) as m7x[e, j, g], y-edges
        # (X_ig, Y_e) as m7y[e, i, g]
        m7x = np.zeros((N + 1, N, me, 7))
        m7y = np.zeros((N + 1, N, me, 7))
        for e in range(N + 1):
            Xe = np.tan(-np.pi / 4 + e * self.dx)
            for j in range(N):
                for g in range(me):
                    Xg = np.tan(-np.pi / 4 + (j + 0.5 + gx[g]) * self.dx)
                    m7x[e, j, g] = O.metric(Xe, Xg)
                    m7y[e, j, g] = O.metric(Xg, Xe)
        self.m7x, self.m7y = torch.tensor(m7x), torch.tensor(m7y)
        # cell points: X, Y and Coriolis parameter per panel
        Xc = np.tan(-np.pi / 4 + (np.arange(N)[:, None] + 0.5 + gx[None, :]) * self.dx)  # (N, me)
        self.Xc = torch.tensor(Xc)
        fcor = np.zeros((6, N, N, me, me))  # [p, j, i, h, g]
        for p in range(6):
            for j in range(N):
                for i in range(N):
                    for h in range(me):
                        for g in range(me):
                            fcor[p, j, i, h, g] = o.coriolis(p, Xc[i, g], Xc[j, h])
        self.fcor = torch.tensor(fcor)
        self.et = o.edge_tables()

    # ------------------------------------------------------------------ pieces
    def fill_ghosts(self, q):
        N, H, ne, me = self.N, self.H, self.ne, self.me
        flat = torch.nn.functional.pad(q, (H, H, H, H)).reshape(3, -1)  # ghosts start at zero
        for _ in range(self.iters):
            vals = (flat[:, self.g_src] * self.g_w).sum(-1)  # (3, nGQP)
            m = self.g_ratio * vals[0]
            u = self.g_C[:, 0] * vals[1] + self.g_C[:, 1] * vals[2]
            v = self.g_C[:, 2] * vals[1] + self.g_C[:, 3] * vals[2]
            gq = torch.stack([m, u, v]).reshape(3, -1, me * me, 2).sum(-1)
            ghost = (gq * self.g_W).sum(-1)  # (3, 6*nring)
            flat = flat.clone()
            flat[:, self.ring_idx] = ghost
        return flat.reshape(3, 6, ne, ne)

    def reconstruct(self, ext):
        """(3, 6*N*N, npoc) point values."""
        st = ext.reshape(3, -1)[:, self.st_idx]  # (3, ncell, K*K)
        if self.scheme == O.TPP:
            return st @ self.R.T
        sub = st[:, :, self.sub_idx]  # (3, ncell, s, l*l)
        p = torch.einsum("vcsl,psl->vcps", sub, self.rsub)
        beta = torch.einsum("vcsl,slm,vcsm->vcs", sub, self.M, sub)
        s = self.s
        diff = (beta[..., :, None] - beta[..., None, :]).abs()
        iu = torch.triu_indices(s, s, offset=0)
        tau = 2.0 / ((s + 1) * s) * diff[..., iu[0], iu[1]].sum(-1)  # pairs eta <= psi
        f = 1.0 + tau[..., None] / (beta + self.eps)  # (3, ncell, s)
        ap = (self.gp / self.sp[:, None])[None, None] * f[:, :, None, :]
        am = (self.gm / self.sm[:, None])[None, None] * f[:, :, None, :]
        wp = ap / ap.sum(-1, keepdim=True)
        wm = am / am.sum(-1, keepdim=True)
        return self.sp * (wp * p).sum(-1) - self.sm * (wm * p).sum(-1)

    def lmars(self, d, m7, qL, qR):
        r2 = self.r ** 2
        sG = m7[..., 0]
        Gii = (m7[..., 1] if d == 0 else m7[..., 3]) / r2
        G1i = (m7[..., 1] if d == 0 else m7[..., 2]) / r2
        G2i = (m7[..., 2] if d == 0 else m7[..., 3]) / r2
        phL, phR = qL[0] / sG, qR[0] / sG
        uL = qL[1 + d] / qL[0] / torch.sqrt(Gii)
        uR = qR[1 + d] / qR[0] / torch.sqrt(Gii)
        c = 0.5 * (torch.sqrt(phL) + torch.sqrt(phR))
        ms = 0.5 * (uL + uR - (phR - phL) / c)
        ph = 0.5 * (phL + phR - c * (uR - uL))
        m = ms * torch.sqrt(Gii)
        F = 0.5 * (m * (qL + qR) - m.abs() * (qR - qL))
        P = torch.stack([torch.zeros_like(ph), 0.5 * sG * G1i * ph ** 2, 0.5 * sG * G2i * ph ** 2])
        return F + P

    def tendency(self, q):
        N, me, dx = self.N, self.me, self.dx
        ext = self.fill_ghosts(q)
        P = self.reconstruct(ext).reshape(3, 6, N, N, self.npoc)
        W_, E_, S_, N_ = (slice(s * me, (s + 1) * me) for s in range(4))
        gw = self.gw
        # interior x-edges (between cells e-1 and e), F at (p, j, e, g)
        qL = P[:, :, :, :-1, E_]
        qR = P[:, :, :, 1:, W_]
        m7x = self.m7x[1:N].permute(1, 0, 2, 3)[None]  # (1, j, e, g, 7)
        Fx_in = (self.lmars(0, m7x, qL, qR) * gw).sum(-1)  # (3, 6, N, N-1)
        # interior y-edges (cells e-1 | e in column i)
        qL = P[:, :, :-1, :, N_]
        qR = P[:, :, 1:, :, S_]
        m7y = self.m7y[1:N][None]  # (1, e, i, g, 7)
        Fy_in = (self.lmars(1, m7y, qL, qR) * gw).sum(-1)  # (3, 6, N-1, N)
        zx = torch.zeros(3, 6, N, 1, dtype=q.dtype)
        zy = torch.zeros(3, 6, 1, N, dtype=q.dtype)
        Fx = torch.cat([zx, Fx_in, zx], dim=-1)  # boundary columns set below
        Fy = torch.cat([zy, Fy_in, zy], dim=2)
        # panel-boundary edges: single flux per shared point, in the lower panel's frame
        et = self.et
        for A in range(6):
            for side in range(4):
                base = ((A * 4 + side) * N) * me
                B = int(et["B"][base])
                if B < A:
                    continue
                sideB = int(et["sideB"][base])
                sA = 1.0 if side in (1, 3) else -1.0
                sB = 1.0 if sideB in (1, 3) else -1.0
                rows = np.arange(N * me) + base
                t = np.repeat(np.arange(N), me)
                g = np.tile(np.arange(me), N)
                tB, gB = et["tB"][rows], et["gB"][rows]
                ci = {0: np.zeros(N * me, int), 1: np.full(N * me, N - 1)}.get(side, t)
                cj = {2: np.zeros(N * me, int), 3: np.full(N * me, N - 1)}.get(side, t)
                bi = {0: np.zeros(N * me, int), 1: np.full(N * me, N - 1)}.get(sideB, tB)
                bj = {2: np.zeros(N * me, int), 3: np.full(N * me, N - 1)}.get(sideB, tB)
                qin = P[:, A, cj, ci, side * me + g]  # (3, N*me)
                qb = P[:, B, bj, bi, sideB * me + gB]
                ratio = torch.tensor(et["ratio"][rows])
                C = torch.tensor(et["C"][rows])
                qo = torch.stack([ratio * qb[0], C[:, 0] * qb[1] + C[:, 1] * qb[2], C[:, 2] * qb[1] + C[:, 3] * qb[2]])
                dirA = side // 2
                e = N if side in (1, 3) else 0
                m7 = (self.m7x if dirA == 0 else self.m7y)[e, t, g]  # (N*me, 7)
                F = self.lmars(dirA, m7, qin, qo) if sA > 0 else self.lmars(dirA, m7, qo, qin)
                w = gw[g]
                FA = (F * w).reshape(3, N, me).sum(-1)
                det = C[:, 0] * C[:, 3] - C[:, 1] * C[:, 2]
                Ci = torch.stack([C[:, 3], -C[:, 1], -C[:, 2], C[:, 0]], 1) / det[:, None]
                sg = -sA * sB
                FBm = sg * torch.stack([Ci[:, 0] * F[1] + Ci[:, 1] * F[2], Ci[:, 2] * F[1] + Ci[:, 3] * F[2]])
                # B's momentum quadrature in B's node order; B's mass flux is A's, signed
                FBm_o = torch.zeros(2, N, me, dtype=q.dtype)
                FBm_o = FBm_o.index_put((torch.arange(2)[:, None], torch.tensor(tB)[None], torch.tensor(gB)[None]), FBm)
                FBq = (FBm_o * gw).sum(-1)  # (2, N) indexed by B's cell
                tBc = tB.reshape(N, me)[:, 0]
                FB0 = torch.zeros(N, dtype=q.dtype).index_put((torch.tensor(tBc),), sg * FA[0])
                FBall = torch.cat([FB0[None], FBq], 0)  # (3, N) indexed by B's cell
                if dirA == 0:
                    Fx = Fx.clone()
                    Fx[:, A, :, e] = FA
                else:
                    Fy = Fy.clone()
                    Fy[:, A, e, :] = FA
                eB = N if sideB in (1, 3) else 0
                if sideB // 2 == 0:
                    Fx = Fx.clone()
                    Fx[:, B, :, eB] = FBall
                else:
                    Fy = Fy.clone()
                    Fy[:, B, eB, :] = FBall
        # sources at the cell points
        cq = P[..., 4 * me:].reshape(3, 6, N, N, me, me)  # [..., h, g]
        X = self.Xc[None, None, :, None, :].expand(6, N, N, me, me)  # x node of column i, g
        Y = self.Xc[None, :, None, :, None].expand(6, N, N, me, me)  # y node of row j, h
        d2 = 1 + X ** 2 + Y ** 2
        sG = (1 + X ** 2) * (1 + Y ** 2) / d2 ** 1.5
        g11 = d2 / (1 + X ** 2)
        g12 = d2 * X * Y / ((1 + X ** 2) * (1 + Y ** 2))
        g22 = d2 / (1 + Y ** 2)
        phi, u, v = cq[0] / sG, cq[1] / cq[0], cq[2] / cq[0]
        pm1 = 2 * sG / d2 * (-X * Y ** 2 * phi * u * u + Y * (1 + Y ** 2) * phi * u * v)
        pm2 = 2 * sG / d2 * (X * (1 + X ** 2) * phi * u * v - X ** 2 * Y * phi * v * v)
        f = self.fcor
        pc1 = sG * f * (-g12 * cq[1] + g11 * cq[2])
        pc2 = sG * f * (-g22 * cq[1] + g12 * cq[2])
        W = torch.outer(self.gw, self.gw)  # [h, g]
        S1 = ((pm1 + pc1) * W).sum((-1, -2))
        S2 = ((pm2 + pc2) * W).sum((-1, -2))
        S = torch.stack([torch.zeros_like(S1), S1, S2])
        return -(Fx[..., 1:] - Fx[..., :-1]) / dx - (Fy[:, :, 1:] - Fy[:, :, :-1]) / dx + S

    def step(self, q, dt):
        q1 = q + dt * self.tendency(q)
        q2 = 0.75 * q + 0.25 * (q1 + dt * self.tendency(q1))
        return q / 3.0 + 2.0 / 3.0 * (q2 + dt * self.tendency(q2))
