"""Oracle: the graph-specific probability density g and its sampler
(Sec. III.A, Eqs. eq_pdf_final and eq_pdf).

TEST INFRASTRUCTURE ONLY (see the package header).

g = C1 g1 + C2 g2 + C3 g3 + C4 g4 on the simplex sum(z) = 1, M = 3n-1.

g1 (Eq. eq_pdf): in the Hepp sector z_{j1} >= ... >= z_{jM}, with
s_l = {j_l, ..., j_M} and t_l = z_{jl}/z_{j(l-1)},
    g1 = C * prod_{l>=2} t_l^Deg(s_l) / prod_i z_i,   C = 1/Phi(all),
where Phi(T) = sum_{j in T} Phi(T\\j)/Deg(T\\j) (|T| >= 2), Phi({j}) = 1.
Because dz delta(1-sum z) = prod(z) prod_{l>=2} dt_l/t_l inside a sector,
g1 is sampled exactly by the sequential walk: from T = all lines remove the
next-largest line j with probability Phi(T\\j)/Deg(T\\j)/Phi(T), and draw
t = u^(1/Deg(T\\j)).

Readings of what the paper leaves to its missing references:
  * Deg(s): d0(s) = n_e(s)/2 + n_gamma(s) - 2 L(s) + 1/2 [merged line in s]
    (power counting in Feynman-parameter units; the merged line is two
    electron propagators).  Deg(s) = d0(s) when d0(s) > 0, otherwise
    1/2 - C_sub with C_sub = C_subI (merged line in s), C_subSE (d0 < 0) or
    C_subO (d0 = 0), constants of Eq. eq_mc_settings; then capped at
    deg_max (default 1): d0 counts only ultraviolet scaling, and where the
    shrinking set is a forest of electron lines the integrand decays only
    like lambda^1 (soft photons in the complement), so a steeper density
    would have infinite variance.  C_bigZ, C_bigF and
    C_add are kept as named parameters; their role is not stated in the
    paper and they are unused.
  * g2 = uniform density (M-1)!; g3 = g1 with Deg -> D*Deg;
    g4 = g1 with Deg -> min(Deg, 1/2).
  * C1..C4, D: Calc 2 values (Sec. V).
The density is kept as log2 (the paper stores x*2^j, Sec. IV.A).

Elementary functions: log2/exp2 are written here from their series
(atanh series for log, Taylor series for exp); the sampler uses Tang's
table-driven forms on tables of those series at the table points, with
plain IEEE multiply, add and divide, so the sample point z is reproducible
bit for bit by any other implementation of the same steps.  The walk
multiplies by 1/Deg and the normalisation by 1/sum (products, not quotients).
The density can be evaluated for the constants of either calculation
(CALC1, CALC2).

Pins: E_g[1/g] = 1/(M-1)! (simplex volume), E_g[z_i/g] = 1/M!, exact
sector probabilities by enumeration for small M.
"""
import math
import numpy as np

C_BIGZ, C_BIGF, C_ADD = 0.256, 0.839, 0.786
C_SUBI, C_SUBSE, C_SUBO = 0.2, 0.0, 0.2
CALC2 = dict(C2=0.03, C3=0.01, C4=0.06, D=0.75)
CALC1 = dict(C2=0.03, C3=0.035, C4=0.035, D=0.75)   # the constants of Calc 1 (Sec. V)

INV_LN2 = 1.4426950408889634
LN2 = 0.6931471805599453
SQRT_HALF = 0.7071067811865476


def log2_series(x):
    """log2 of a positive finite double (numpy array), atanh series."""
    x = np.asarray(x, dtype=np.float64)
    f, k = np.frexp(x)                     # x = f * 2^k, f in [0.5, 1)
    small = f < SQRT_HALF
    f = np.where(small, f * 2.0, f)
    k = np.where(small, k - 1, k).astype(np.float64)
    s = (f - 1.0) / (f + 1.0)
    s2 = s * s
    p = 1.0 / 25.0
    for d in (23.0, 21.0, 19.0, 17.0, 15.0, 13.0, 11.0, 9.0, 7.0, 5.0, 3.0):
        p = p * s2 + 1.0 / d
    p = p * s2 + 1.0
    ln_f = (s + s) * p
    return k + ln_f * INV_LN2


def exp2_series(x):
    """2^x for finite doubles (numpy array), Taylor series of exp."""
    x = np.asarray(x, dtype=np.float64)
    k = np.floor(x + 0.5)
    r = (x - k) * LN2
    p = 1.0 / 6402373705728000.0          # 1/18!
    fact = 6402373705728000.0
    for i in range(18, 0, -1):
        fact = fact / i
        p = p * r + 1.0 / fact
    return np.ldexp(p, k.astype(np.int64))


# Table-driven log2 / exp2 (Tang's method: reduce the argument to a short
# interval around a table point, evaluate a short series there).  The tables
# are the series functions above evaluated at the table points, so they are
# fixed by the same definitions.
#   exp2: x = k/32 + d, |d| <= 1/64:  2^x = 2^(k div 32) * 2^((k mod 32)/32) * exp(d ln 2),
#         exp by its Taylor polynomial of degree 7 (remainder < 5e-21).
#   log2: x = F 2^E with F in [3/4, 3/2); c = j/32 nearest to F (j = 24..48):
#         log2 x = E + log2 c + 2 atanh(s)/ln 2, s = (F - c)/(F + c), |s| <= 1/96,
#         atanh by s (1 + s^2/3 + s^4/5 + s^6/7) (remainder < 2e-19 s).  The
#         interval around 1 keeps log2 x accurate relative to itself near x = 1.
EXP2_TAB = np.array([float(exp2_series(j / 32.0)) for j in range(32)])
LOG2_TAB = np.array([float(log2_series(j / 32.0)) for j in range(24, 49)])


def exp2_tab(x):
    """2^x (numpy array), table-driven; 0 below -1100, inf above 1100, NaN
    for NaN."""
    x0 = np.asarray(x, dtype=np.float64)
    ok = (x0 >= -1100.0) & (x0 <= 1100.0)
    x = np.where(ok, x0, 0.0)
    k = np.floor(x * 32.0 + 0.5)
    m = np.floor(k * 0.03125)
    j = (k - m * 32.0).astype(np.int64)
    r = (x - k * 0.03125) * LN2
    p = 1.0 / 5040.0
    for c in (1.0 / 720.0, 1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 0.5, 1.0, 1.0):
        p = p * r + c
    v = np.ldexp(EXP2_TAB[j] * p, m.astype(np.int64))
    return np.where(ok, v, np.where(x0 > 1100.0, np.inf, np.where(x0 < -1100.0, 0.0, x0)))


def log2_tab(x):
    """log2 (numpy array), table-driven; -inf at 0, inf at inf, NaN for
    negative or NaN arguments."""
    x0 = np.asarray(x, dtype=np.float64)
    ok = (x0 > 0.0) & (x0 < np.inf)
    x = np.where(ok, x0, 1.0)
    f, e = np.frexp(x)                     # x = f * 2^e, f in [0.5, 1)
    low = f < 0.75
    F = np.where(low, f * 2.0, f)
    E = np.where(low, e - 1, e).astype(np.float64)
    jf = np.floor(F * 32.0 + 0.5)
    c = jf * 0.03125
    s = (F - c) / (F + c)
    s2 = s * s
    p = 1.0 / 7.0
    p = p * s2 + 1.0 / 5.0
    p = p * s2 + 1.0 / 3.0
    p = p * s2 + 1.0
    t = ((s + s) * p) * INV_LN2
    v = (E + LOG2_TAB[jf.astype(np.int64) - 24]) + t
    return np.where(ok, v, np.where(x0 == 0.0, -np.inf, np.where(x0 == np.inf, np.inf, np.nan)))


class LineSets:
    """Line structure of one graph in the merged (M = 3n-1) numbering."""

    def __init__(self, g):
        self.g = g
        idx = g.line_index()
        self.M = 3 * g.n - 1
        self.kind = [None] * self.M
        self.ends = [None] * self.M
        for key, i in idx.items():
            if key[0] == 'e':
                if i == 0:
                    self.kind[0] = 'e'
                    self.ends[0] = (g.s - 1, g.s + 1)
                else:
                    self.kind[i] = 'e'
                    self.ends[i] = (key[1] - 1, key[1])
            else:
                self.kind[i] = 'g'
                self.ends[i] = (key[1], key[2])

    def loops(self, mask):
        verts = set()
        ls = [i for i in range(self.M) if mask >> i & 1]
        for i in ls:
            verts.update(self.ends[i])
        par = {v: v for v in verts}

        def f(x):
            while par[x] != x:
                x = par[x]
            return x
        for i in ls:
            a, b = self.ends[i]
            par[f(a)] = f(b)
        comps = len({f(v) for v in verts})
        return len(ls) - len(verts) + comps

    def d0(self, mask):
        ne = sum(1 for i in range(self.M) if mask >> i & 1 and self.kind[i] == 'e')
        ng = sum(1 for i in range(self.M) if mask >> i & 1 and self.kind[i] == 'g')
        return ne / 2.0 + ng - 2.0 * self.loops(mask) + (0.5 if mask & 1 else 0.0)


DEG_MAX = 1.0


def deg_table(g, deg_max=DEG_MAX):
    """Deg(s) for every bitmask s (index 0 and the full set are unused)."""
    ls = LineSets(g)
    M = ls.M
    out = np.zeros(1 << M)
    for s in range(1, (1 << M) - 1):
        d = ls.d0(s)
        if d > 0:
            out[s] = d
        elif s & 1:
            out[s] = 0.5 - C_SUBI
        elif d < 0:
            out[s] = 0.5 - C_SUBSE
        else:
            out[s] = 0.5 - C_SUBO
        if deg_max > 0 and out[s] > deg_max:
            out[s] = deg_max
    return out


def phi_table(deg, M):
    """Phi(T) by the recursion above, summing over j in ascending order."""
    phi = np.zeros(1 << M)
    for T in range(1, 1 << M):
        if T & (T - 1) == 0:
            phi[T] = 1.0
            continue
        acc = 0.0
        for j in range(M):
            if T >> j & 1:
                R = T ^ (1 << j)
                acc = acc + phi[R] / deg[R]
        phi[T] = acc
    return phi


class Density:
    """Tables of the three sector densities g1, g3, g4 of one graph."""

    def __init__(self, g, C2=CALC2['C2'], C3=CALC2['C3'], C4=CALC2['C4'], D=CALC2['D'],
                 deg_max=DEG_MAX):
        self.M = 3 * g.n - 1
        M = self.M
        d1 = deg_table(g, deg_max)
        self.deg = [d1, d1 * D, np.minimum(d1, 0.5)]
        self.phi = [phi_table(d, M) for d in self.deg]
        self.C = [1.0 - C2 - C3 - C4, C3, C4]      # mixture weights of g1, g3, g4
        self.C2 = C2
        self.full = (1 << M) - 1
        self.log2_fact = float(log2_tab(float(math.factorial(M - 1))))  # log2 (M-1)!


def sample(dens, u):
    """Draw samples from g.  u: (S, >= 2M) uniforms in (0,1), consumed as
    u[:,0] = component pick; sector walk: u[:,1+2l] = choice, u[:,2+2l] = t;
    uniform component: u[:,1+i], i < M.
    Returns (z, log2g, comp)."""
    M = dens.M
    S = u.shape[0]
    pick = u[:, 0]
    c1, c3, c4 = dens.C
    # cumulative in the order g1, g2, g3, g4
    comp = np.where(pick < c1, 0,
           np.where(pick < c1 + dens.C2, 1,
           np.where(pick < c1 + dens.C2 + c3, 2, 3)))
    lz = np.zeros((S, M))
    zz = np.zeros((S, M))
    for ci, k in ((0, 0), (2, 1), (3, 2)):
        sel = np.nonzero(comp == ci)[0]
        if sel.size == 0:
            continue
        deg, phi = dens.deg[k], dens.phi[k]
        with np.errstate(divide="ignore"):
            dinv = 1.0 / deg    # the empty and the full set (Deg 0) are never used
        T = np.full(sel.size, dens.full, dtype=np.int64)
        cur = np.zeros(sel.size)
        for l in range(M - 1):
            uc = u[sel, 1 + 2 * l]
            ut = u[sel, 2 + 2 * l]
            target = uc * phi[T]
            acc = np.zeros(sel.size)
            chosen = np.full(sel.size, -1, dtype=np.int64)
            for j in range(M):
                has = (T >> j & 1) == 1
                R = T ^ (1 << j)
                acc = np.where(has, acc + phi[np.where(has, R, 1)] / deg[np.where(has, R, 1)], acc)
                newly = has & (chosen < 0) & (target < acc)
                chosen = np.where(newly, j, chosen)
            # guard against rounding at the top end: take the last member
            last = np.zeros(sel.size, dtype=np.int64)
            for j in range(M):
                last = np.where(T >> j & 1 == 1, j, last)
            chosen = np.where(chosen < 0, last, chosen)
            lz[sel, chosen] = cur
            T = T ^ (np.int64(1) << chosen)
            cur = cur + log2_tab(ut) * dinv[T]   # log2 t = log2(u) * (1/Deg)
        # the last remaining line
        lastj = np.zeros(sel.size, dtype=np.int64)
        for j in range(M):
            lastj = np.where(T >> j & 1 == 1, j, lastj)
        lz[sel, lastj] = cur
        e = exp2_tab(lz[sel])
        ssum = np.zeros(sel.size)
        for i in range(M):
            ssum = ssum + e[:, i]
        zz[sel] = e * (1.0 / ssum)[:, None]
        lz[sel] = lz[sel] - log2_tab(ssum)[:, None]
    sel = np.nonzero(comp == 1)[0]
    if sel.size:
        L = -log2_tab(u[sel, 1:1 + M])
        ssum = np.zeros(sel.size)
        for i in range(M):
            ssum = ssum + L[:, i]
        zz[sel] = L * (1.0 / ssum)[:, None]
        lz[sel] = log2_tab(L) - log2_tab(ssum)[:, None]
    return zz, log2_density(dens, lz), comp


def sector_order(lz):
    """Descending order of log2 z, ties by lower index (stable)."""
    return np.argsort(-lz, axis=1, kind='stable')


def log2_density(dens, lz):
    """log2 g at points given by log2 z (S, M)."""
    M = dens.M
    S = lz.shape[0]
    order = sector_order(lz)
    sumlz = np.zeros(S)
    for i in range(M):
        sumlz = sumlz + lz[:, i]
    terms = []
    for k in range(3):
        deg, phi = dens.deg[k], dens.phi[k]
        acc = np.zeros(S)
        T = np.full(S, dens.full, dtype=np.int64)
        rows = np.arange(S)
        prev = lz[rows, order[:, 0]]
        T = T ^ (np.int64(1) << order[:, 0])
        for l in range(1, M):
            cur = lz[rows, order[:, l]]
            acc = acc + deg[T] * (cur - prev)
            prev = cur
            T = T ^ (np.int64(1) << order[:, l])
        terms.append(log2_tab(dens.C[k]) - log2_tab(phi[dens.full]) + acc - sumlz)
    terms.insert(1, np.full(S, log2_tab(dens.C2) + dens.log2_fact))
    terms = np.stack(terms, 1)
    m = terms.max(1)
    rel = np.zeros(S)
    for k in range(4):
        rel = rel + exp2_tab(terms[:, k] - m)
    return m + log2_tab(rel)
