"""A second, independent restatement of the SLPIC-MCC step in pure Python, for
brute-force checks of the oracle on a handful of markers.

It is written differently from the oracle on purpose: positions are continuous
coordinates x in [0, d) instead of (cell, offset) pairs, Philox is computed
with Python integers, the field solve is a dense linear solve (numpy), and the
loop structure follows the method's step order directly.  FP64 throughout.
"""
import math

import numpy as np

QE = 1.602176634e-19
ME = 9.1093837015e-31
KB = 1.380649e-23
EPS0 = 8.8541878128e-12
GEN = 0x80000000
MASK32 = 0xFFFFFFFF


def philox(c, key):
    """Philox4x32-10 on a list of four 32-bit words with a 64-bit key."""
    c = list(c)
    k0, k1 = key & MASK32, (key >> 32) & MASK32
    for r in range(10):
        if r:
            k0 = (k0 + 0x9E3779B9) & MASK32
            k1 = (k1 + 0xBB67AE85) & MASK32
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & MASK32, p1 & MASK32,
             ((p0 >> 32) ^ c[3] ^ k1) & MASK32, p0 & MASK32]
    return c


def philox2(c, key):
    """Philox2x32-10 on two 32-bit words with a 32-bit key."""
    c0, c1 = c
    k = key & MASK32
    for r in range(10):
        if r:
            k = (k + 0x9E3779B9) & MASK32
        p = 0xD256D193 * c0
        c0, c1 = ((p >> 32) ^ c1 ^ k) & MASK32, p & MASK32
    return [c0, c1]


def unif(x):
    return ((x >> 9) + 0.5) / 8388608.0


class ScalarSim:
    def __init__(self, spec):
        s = spec
        self.s = s
        self.N = s["n_cells"]
        self.d = s["d"]
        self.dx = s["d"] / s["n_cells"]
        self.dt = s["dt"]
        self.ng = s["p_Pa"] / (KB * s["T_K"])
        self.m = [s["mass_e"], s["mass_i"]]
        self.q = [s["charge_e"], s["charge_i"]]
        self.vl = [s["vlim_e"], s["vlim_i"]]
        self.E = np.full(self.N + 1, -s["V"] / s["d"])
        L, sub, octv = s["tab_lo_exp2"], s["tab_log2_sub"], s["tab_octaves"]
        self.L, self.sub, self.oct = L, sub, octv
        el = s["sig_el"].astype(np.float64)
        ex = s["sig_ex"].astype(np.float64)
        io = s["sig_io"].astype(np.float64)
        self.tab = [el, el + ex, el + ex + io]
        self.smax = float(np.max(self.tab[2]))
        etop = math.ldexp(1.0, L + octv)
        vtop = math.sqrt(etop * (2.0 * QE / ME))
        vl = self.vl[0] if math.isfinite(self.vl[0]) and self.vl[0] > 0 else math.inf
        self.vbcap = min(vl, vtop)
        self.ndt = self.ng * self.dt
        self.P0 = (self.ndt * self.vbcap) * self.smax
        self.parts = [[], []]  # [x, vx, vy, vz, wj, id]
        self.next_id = [0, 0]
        self.step_no = 0
        self.hist = []

    def beta(self, v, sp):
        vl = self.vl[sp]
        if not (vl > 0 and math.isfinite(vl)):
            return 1.0
        return vl / v if v > vl else 1.0

    def kick(self, vx, vy, vz, A, sp):
        """v_x after one step's kick, A = q E dt / m (Eq. slpicEOMv with the
        field held over the step).  In the time tau = integral of beta dt the
        motion is unlimited, v_x(tau) = vx + (A / dt) tau, and the step's
        elapsed time is the integral of 1 / beta(|v(tau)|) dtau.  The end is
        the tau in [0, dt] where that integral reaches dt: the integral is
        taken by adaptive quadrature (split where the speed crosses the limit,
        where the integrand has a kink) and the root by Brent's method."""
        L = self.vl[sp]
        if not (L > 0 and math.isfinite(L)):
            return vx + A
        if A == 0.0:
            return vx
        from scipy import integrate, optimize
        perp2 = vy * vy + vz * vz
        dt = 1.0
        a = A / dt

        def inv_beta(tau):
            u = vx + a * tau
            return max(1.0, math.sqrt(u * u + perp2) / L)

        # the speed crosses L where (vx + a tau)^2 = L^2 - perp2
        kinks = []
        if perp2 < L * L:
            q = math.sqrt(L * L - perp2)
            kinks = sorted(t for t in ((q - vx) / a, (-q - vx) / a) if 0.0 < t < dt)

        def elapsed(tau):
            pts = [0.0] + [k for k in kinks if k < tau] + [tau]
            return sum(integrate.quad(inv_beta, x0, x1, epsabs=0.0, epsrel=1e-13, limit=200)[0]
                       for x0, x1 in zip(pts[:-1], pts[1:]))

        if elapsed(dt) <= dt * (1.0 + 1e-15):
            return vx + A
        tau = optimize.brentq(lambda t: elapsed(t) - dt, 0.0, dt, xtol=1e-16 * dt,
                              rtol=1e-15, maxiter=200)
        return vx + a * tau

    def draws(self, ident, step, sp, blk):
        c = [ident, step & MASK32, (self.s.get("instance", 0) * 2 + sp) & MASK32, blk]
        return [unif(w) for w in philox(c, self.s["seed"])]

    def sig(self, eps):
        lo = math.ldexp(1.0, self.L)
        hi = math.ldexp(1.0, self.L + self.oct)
        n_last = (self.oct << self.sub)
        if not eps >= lo:
            j, t = 0, 0.0
        elif eps >= hi:
            j, t = n_last, 0.0
        else:
            m, e = math.frexp(eps)
            pos = (2.0 * m - 1.0) * (1 << self.sub)
            j = ((e - 1 - self.L) << self.sub) + int(math.floor(pos))
            t = pos - math.floor(pos)
        out = []
        for T in self.tab:
            a = T[j]
            b = T[min(j + 1, n_last)]
            out.append(a + t * (b - a))
        return out

    @staticmethod
    def iso(speed, ua, ub):
        ct = 1.0 - 2.0 * ua
        st = math.sqrt(max(0.0, (1.0 - ct) * (1.0 + ct)))
        ph = 2.0 * math.pi * ub
        return speed * ct, speed * st * math.cos(ph), speed * st * math.sin(ph)

    def step(self):
        stp = self.step_no
        born_e, born_see, born_i = [], [], []
        tally = {"n_abs": [[0, 0], [0, 0]], "n_coll": [0, 0, 0], "n_see": 0}
        for sp in (0, 1):
            keep = []
            for (x, vx, vy, vz, wj, ident) in self.parts[sp]:
                k = min(int(math.floor(x / self.dx)), self.N - 1)
                f = x / self.dx - k
                Ex = self.E[k] * (1.0 - f) + self.E[k + 1] * f
                a = self.q[sp] / self.m[sp] * Ex
                vx = self.kick(vx, vy, vz, a * self.dt, sp)
                v1 = math.sqrt(vx * vx + vy * vy + vz * vz)
                x += self.beta(v1, sp) * vx * self.dt
                if x < 0.0:
                    tally["n_abs"][sp][0] += 1
                    if sp == 1:
                        u = self.draws(ident, stp, 1, 0)
                        if u[0] < self.s["gamma_se"]:
                            born_see.append([0.0, 0.0, 0.0, 0.0, wj, GEN])
                            tally["n_see"] += 1
                    continue
                if x >= self.d:
                    tally["n_abs"][sp][1] += 1
                    continue
                if sp == 0:
                    seed = self.s["seed"]
                    key2 = ((seed & MASK32) ^ (seed >> 32) ^ (0x85EBCA6B * (self.s.get("instance", 0) + 1))) & MASK32
                    u1 = unif(philox2([ident, stp & MASK32], key2)[0])
                    u = self.draws(ident, stp, 0, 0)
                    if u1 < self.P0:
                        vl = self.vl[0] if (self.vl[0] > 0 and math.isfinite(self.vl[0])) else math.inf
                        vb = min(min(v1, vl), self.vbcap)
                        eps = 0.5 * ME * v1 * v1 / QE
                        s1, s2, s3 = self.sig(eps)
                        r = u[1] * self.P0
                        c = self.ndt * vb
                        proc = 0 if r < c * s1 else 1 if r < c * s2 else 2 if r < c * s3 else 3
                        if proc < 3:
                            tally["n_coll"][proc] += 1
                        kv = 2.0 * QE / ME
                        if proc == 0:
                            cc = (2.0 + eps - 2.0 * (1.0 + eps) ** u[2]) / eps
                            cc = min(1.0, max(-1.0, cc))
                            chi = math.acos(cc)
                            ph = 2.0 * math.pi * u[3]
                            e_new = eps * (1.0 - 2.0 * ME / self.m[1] * (1.0 - cc))
                            uvec = np.array([vx, vy, vz]) / v1
                            # rotation via an explicit orthonormal frame
                            ref = np.array([1.0, 0.0, 0.0]) if abs(uvec[0]) <= 0.99 else np.array([0.0, 0.0, 1.0])
                            e1 = ref - np.dot(ref, uvec) * uvec
                            e1 /= np.linalg.norm(e1)
                            e2 = np.cross(uvec, e1)
                            nv = (math.cos(chi) * uvec + math.sin(chi) * (math.cos(ph) * e1 + math.sin(ph) * e2))
                            vx, vy, vz = (math.sqrt(e_new * kv) * nv).tolist()
                        elif proc == 1:
                            vx, vy, vz = self.iso(math.sqrt(max(0.0, eps - self.s["e_ex"]) * kv), u[2], u[3])
                        elif proc == 2:
                            eav = max(0.0, eps - self.s["e_io"])
                            b = self.draws(ident, stp, 0, 1)
                            es = b[0] * eav
                            vx, vy, vz = self.iso(math.sqrt((eav - es) * kv), u[2], u[3])
                            bx, by, bz = self.iso(math.sqrt(es * kv), b[1], b[2])
                            born_e.append([x, bx, by, bz, wj, ident & GEN])
                            g = self.draws(ident, stp, 0, 2)
                            sT = math.sqrt(KB * self.s["T_K"] / self.m[1])
                            r1 = math.sqrt(-2.0 * math.log(g[0]))
                            r2 = math.sqrt(-2.0 * math.log(g[2]))
                            born_i.append([x, sT * r1 * math.cos(2 * math.pi * g[1]),
                                           sT * r1 * math.sin(2 * math.pi * g[1]),
                                           sT * r2 * math.cos(2 * math.pi * g[3]), wj, ident & GEN])
                keep.append([x, vx, vy, vz, wj, ident])
            self.parts[sp] = keep
        for lst, sp in ((born_e, 0), (born_see, 0), (born_i, 1)):
            for p in lst:
                p[5] = (p[5] & GEN) | self.next_id[sp]
                self.next_id[sp] += 1
                self.parts[sp].append(p)
        # deposit (fixed point, 24-bit linear weights) and field solve
        self.charge = []
        for sp in (0, 1):
            q = np.zeros(self.N + 1, dtype=object)
            for (x, vx, vy, vz, wj, ident) in self.parts[sp]:
                v = math.sqrt(vx * vx + vy * vy + vz * vz)
                Q = int(round(self.beta(v, sp) * wj * 2.0 ** self.s["charge_shift"]))
                k = min(int(math.floor(x / self.dx)), self.N - 1)
                f = int((x / self.dx - k) * 16777216.0)
                right = (Q * f) >> 24
                q[k] += Q - right
                q[k + 1] += right
            self.charge.append(np.array(q, dtype=np.int64))
        if self.s.get("field_mode", 0) == 1:
            self.solve()
        tally["n_live"] = [len(self.parts[0]), len(self.parts[1])]
        self.hist.append(tally)
        self.step_no += 1

    def solve(self):
        N, dx = self.N, self.dx
        net = (self.charge[1] - self.charge[0]).astype(np.float64)
        rho = QE * net * 2.0 ** (-self.s["charge_shift"]) / (self.s["area"] * dx)
        A = np.zeros((N - 1, N - 1))
        b = -rho[1:N] * dx * dx / EPS0
        for i in range(N - 1):
            A[i, i] = -2.0
            if i > 0:
                A[i, i - 1] = 1.0
            if i < N - 2:
                A[i, i + 1] = 1.0
        b[-1] -= self.s["V"]
        phi = np.concatenate([[0.0], np.linalg.solve(A, b), [self.s["V"]]])
        E = np.empty(N + 1)
        E[1:N] = -(phi[2:] - phi[:-2]) / (2 * dx)
        E[0] = -(phi[1] - phi[0]) / dx
        E[N] = -(phi[N] - phi[N - 1]) / dx
        self.E = E
        self.phi = phi
