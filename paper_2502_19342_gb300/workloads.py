"""Seeded synthetic workloads: meshes, degree / FV patterns and initial states.

This module only builds inputs.  It holds no step of the right-hand side: the
one piece of physics here is the ideal-gas mixture relation used to turn an
initial (rho_k, v, p) field into conserved variables, which is how each
workload's initial condition is specified.  It is shared by the tests, the
benchmark and the CPU oracle's callers; it imports neither the CUDA binding
nor the oracle.

A *problem* is a plain dict (see ``make_problem``); states are flat float64
arrays in the element-contiguous layout

    U[off_e + v*n^3 + i + n*(j + n*k)],  n = N_e+1 (DG) or n_fv (FV),

with variables (rho_1..rho_Nk, rho v_x, rho v_y, rho v_z, rho E) and elements
ordered domain by domain, x fastest.
"""
import math

import numpy as np

# Universal gas constant in the nondimensional units of every workload.
R_UNIVERSAL = 1.0

AIR = dict(gamma=1.4, M=29.0)
HEAVY = dict(gamma=1.249, M=3.5 * 29.0)  # density ratio 3.5 to air at equal p, T
CO2 = dict(gamma=1.3, M=44.0)
HELIUM = dict(gamma=1.67, M=4.0)


def species_set(specs, mu=0.0, Pr=0.72, Sc=1.0, rho_ref=1.0):
    """Species property arrays; D_k = mu / (Sc rho_ref) (constant, Sec. 2)."""
    n = len(specs)
    return dict(
        gamma=np.array([s["gamma"] for s in specs], float),
        Rgas=np.array([R_UNIVERSAL / s["M"] for s in specs], float),
        mu=np.full(n, float(mu)),
        Pr=np.full(n, float(Pr)),
        Dk=np.full(n, float(mu) / (Sc * rho_ref)),
    )


def make_problem(domains, species, n_fv, N, fv=None, riemann=0, nodes=0, split=0, chain=0, fv_own_n=0):
    """domains: list of (dims(3), lo(3), hi(3)); species: dict from species_set;
    nodes 0 = Legendre-Gauss, 1 = Legendre-Gauss-Lobatto; split 1 = split-form
    volume integral (LGL only); chain 1 = the domains glued in order along x
    (conforming or mortar interfaces between neighbours, Sec. 3.2.3)."""
    dims = np.array([d[0] for d in domains], np.int32).reshape(-1, 3)
    lo = np.array([d[1] for d in domains], float).reshape(-1, 3)
    hi = np.array([d[2] for d in domains], float).reshape(-1, 3)
    n_elem = int(np.prod(dims, axis=1).sum())
    N = np.broadcast_to(np.asarray(N, np.int8), (n_elem,)).copy()
    fv = np.zeros(n_elem, np.uint8) if fv is None else np.broadcast_to(np.asarray(fv, np.uint8), (n_elem,)).copy()
    p = dict(dims=dims, lo=lo, hi=hi, n_fv=int(n_fv), riemann=int(riemann), N=N, fv=fv, nodes=int(nodes),
             split=int(split), chain=int(chain), fv_own_n=int(fv_own_n))
    p.update({k: np.array(v, float) for k, v in species.items()})
    return p


def chain_domains(segments, L=(1.0, 1.0)):
    """Domains of a chain along x: segments = [(nx, ny, nz, x_length), ...] placed
    one after the other from x = 0, all on [0, L_y] x [0, L_z].  Neighbouring
    segments need equal ny, nz, or twice as many in one or both (mortar types 1-3,
    Sec. 3.2.3)."""
    out, x0 = [], 0.0
    for nx, ny, nz, lx in segments:
        out.append(((nx, ny, nz), (x0, 0.0, 0.0), (x0 + lx, L[0], L[1])))
        x0 += lx
    return out


def n_elements(prob):
    return int(np.prod(prob["dims"], axis=1).sum())


def n_vars(prob):
    return len(prob["gamma"]) + 4


def points_per_dir(prob):
    """Points per direction: N+1 for DG elements; for FV elements n_fv, or N+1
    when every FV element has its own count (fv_own_n)."""
    n_fv = prob["N"].astype(np.int64) + 1 if prob.get("fv_own_n", 0) else prob["n_fv"]
    return np.where(prob["fv"] != 0, n_fv, prob["N"].astype(np.int64) + 1)


def offsets(prob):
    n = points_per_dir(prob)
    sizes = n_vars(prob) * n ** 3
    off = np.zeros(len(n), np.int64)
    off[1:] = np.cumsum(sizes)[:-1]
    return off, int(sizes.sum())


def n_dofs(prob):
    """Degrees of freedom: nodes of DG elements plus sub-cells of FV elements."""
    return int((points_per_dir(prob) ** 3).sum())


def element_index(prob):
    """Per element: domain id, integer position (3), lower corner (3), size h (3)."""
    dom, pos, corner, h = [], [], [], []
    for d, (dm, lo, hi) in enumerate(zip(prob["dims"], prob["lo"], prob["hi"])):
        nx, ny, nz = (int(x) for x in dm)
        hd = (hi - lo) / dm
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
        dom.append(np.full(len(ijk), d))
        pos.append(ijk)
        corner.append(lo + ijk * hd)
        h.append(np.broadcast_to(hd, ijk.shape))
    return np.concatenate(dom), np.concatenate(pos), np.concatenate(corner), np.concatenate(h)


def lgl_nodes(n):
    """Legendre-Gauss-Lobatto points of n = N+1 nodes: -1, the roots of P_N'
    (numpy's Legendre series), +1."""
    N = n - 1
    inner = np.polynomial.legendre.Legendre.basis(N).deriv().roots() if N > 1 else np.zeros(0)
    return np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])


def dg_points(n, nodes=0):
    """DG nodes of one direction: LG (numpy's Gauss-Legendre rule) or LGL."""
    return lgl_nodes(n) if nodes == 1 else np.polynomial.legendre.leggauss(n)[0]


def _ref_points(n, is_fv, nodes=0):
    """Reference coordinates of the points of one direction: DG nodes for DG,
    sub-cell centres for FV."""
    if is_fv:
        return -1.0 + (np.arange(n) + 0.5) * (2.0 / n)
    return dg_points(n, nodes)


def build_state(prob, prim_fn, chunk=4096):
    """Evaluate prim_fn(x, y, z) -> (rho_k list, (vx, vy, vz), p) at every point
    and convert to the conserved variables with the ideal-gas mixture law
    (rho E = p / (kappa_mix - 1) + rho |v|^2 / 2)."""
    nk = len(prob["gamma"])
    V = nk + 4
    cv = prob["Rgas"] / (prob["gamma"] - 1.0)
    cp = prob["gamma"] * cv
    off, size = offsets(prob)
    U = np.zeros(size)
    _, _, corner, h = element_index(prob)
    npd = points_per_dir(prob)
    fv = prob["fv"] != 0
    for n in np.unique(npd):
        for isfv in (False, True):
            sel = np.nonzero((npd == n) & (fv == isfv))[0]
            if len(sel) == 0:
                continue
            r = _ref_points(int(n), isfv, int(prob.get("nodes", 0)))
            kk, jj, ii = np.meshgrid(r, r, r, indexing="ij")
            ref = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)  # (n^3, 3), x fastest
            for s in range(0, len(sel), chunk):
                es = sel[s:s + chunk]
                X = corner[es][:, None, :] + (ref[None, :, :] + 1.0) * 0.5 * h[es][:, None, :]
                rk, vel, p = prim_fn(X[..., 0], X[..., 1], X[..., 2])
                rk = [np.broadcast_to(q, X.shape[:2]) for q in rk]
                vel = [np.broadcast_to(q, X.shape[:2]) for q in vel]
                p = np.broadcast_to(p, X.shape[:2])
                rho = sum(rk)
                cvm = sum(rk[k] * cv[k] for k in range(nk)) / rho
                cpm = sum(rk[k] * cp[k] for k in range(nk)) / rho
                kap = cpm / cvm
                fields = list(rk) + [rho * vel[0], rho * vel[1], rho * vel[2],
                                     p / (kap - 1.0) + 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)]
                blk = np.stack(fields, axis=1)  # (ne, V, n^3)
                n3 = int(n) ** 3
                idx = off[es][:, None] + np.arange(V * n3)[None, :]
                U[idx.ravel()] = blk.reshape(len(es), V * n3).ravel()
    return U


def constant_state(prob, rho_k, v, p):
    return build_state(prob, lambda x, y, z: ([np.full(x.shape, r) for r in rho_k], v, np.full(x.shape, p)))


# ----------------------------------------------------------------- random patterns
def random_degrees(n_elem, lo, hi, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=n_elem).astype(np.int8)


def random_fv(n_elem, frac, seed):
    rng = np.random.default_rng(seed + 7919)
    return (rng.random(n_elem) < frac).astype(np.uint8)


def smooth_random_state(prob, seed, amp=0.05, rho0=1.0, p0=1.0, vel=(0.3, -0.2, 0.1)):
    """Smooth periodic random-phase state (low Fourier modes of the first domain's
    box, or of the whole chain when the domains are glued along x)."""
    rng = np.random.default_rng(seed + 104729)
    nk = len(prob["gamma"])
    modes = [(a, b, c) for a in range(0, 2) for b in range(0, 2) for c in range(0, 2) if (a, b, c) != (0, 0, 0)]
    ph = rng.uniform(0, 2 * np.pi, size=(6, len(modes)))
    if prob.get("chain", 0):
        lo0, hi0 = np.min(prob["lo"], axis=0), np.max(prob["hi"], axis=0)
    else:
        lo0, hi0 = prob["lo"][0], prob["hi"][0]
    L = hi0 - lo0

    def wave(x, y, z, q):
        s = 0.0
        for m, (a, b, c) in enumerate(modes):
            s = s + np.cos(2 * np.pi * (a * (x - lo0[0]) / L[0] + b * (y - lo0[1]) / L[1] + c * (z - lo0[2]) / L[2]) + ph[q, m])
        return s / len(modes)

    def fn(x, y, z):
        Y1 = 0.5 + 0.3 * wave(x, y, z, 0)
        fr = [Y1] + [(1.0 - Y1) / (nk - 1)] * (nk - 1) if nk > 1 else [1.0 + 0 * x]
        rho = rho0 * (1.0 + amp * wave(x, y, z, 1))
        rk = [rho * f for f in fr]
        v = [vel[i] + amp * wave(x, y, z, 2 + i) for i in range(3)]
        p = p0 * (1.0 + amp * wave(x, y, z, 5))
        return rk, v, p

    return build_state(prob, fn)


# ----------------------------------------------------------------- paper-shaped workloads
def plain_tiny(seed=0, riemann=0):
    """3D periodic [0,1]^3, 4x4x4 elements, uniform N=3, two species
    (gamma 1.4 / M 29 and gamma 1.67 / M 4), viscosity 1e-3, Pr 0.72, Sc 1.
    Uniform velocity (1, 0.5, 0.25) at p = 1, Y_1 = 0.5 + 0.4 sin(2 pi x) sin(2 pi y),
    density 1 + 1e-3 * (8 random-phase cosine modes)."""
    sp = species_set([AIR, HELIUM], mu=1e-3, Pr=0.72, Sc=1.0)
    prob = make_problem([((4, 4, 4), (0, 0, 0), (1, 1, 1))], sp, n_fv=4, N=3, riemann=riemann)
    rng = np.random.default_rng(seed)
    ks = [(a, b, c) for a in (1, 2) for b in (1, 2) for c in (1, 2)]
    ph = rng.uniform(0, 2 * np.pi, len(ks))

    def fn(x, y, z):
        Y1 = 0.5 + 0.4 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
        rho = 1.0 + 1e-3 * sum(np.cos(2 * np.pi * (a * x + b * y + c * z) + ph[m]) for m, (a, b, c) in enumerate(ks))
        return [rho * Y1, rho * (1 - Y1)], (1.0, 0.5, 0.25), np.ones_like(x)

    return prob, build_state(prob, fn)


SHOCK_MACH = 1.5


def _post_shock(gamma, Ms, rho1=1.0, p1=1.0):
    """Rankine-Hugoniot state behind a shock of Mach Ms moving into gas at rest."""
    r = (gamma + 1) * Ms ** 2 / ((gamma - 1) * Ms ** 2 + 2)
    pr = 1 + 2 * gamma / (gamma + 1) * (Ms ** 2 - 1)
    c1 = math.sqrt(gamma * p1 / rho1)
    u2 = Ms * c1 * (1 - 1 / r)
    return rho1 * r, p1 * pr, u2


def hp_shock(seed=0, nel=(16, 16, 16), riemann=0, mu=1e-4, y_bg=0.0, perturb=0.0):
    """[0,2]x[0,1]x[0,1], periodic, 16^3 elements, N drawn from {2..6},
    N_FV = 7; a Mach 1.5 planar shock in air at x = 0.4 moving +x towards a
    bubble (r = 0.2, centre (0.8, 0.5, 0.5)) of the heavy species (density
    ratio 3.5), interface smoothed over 2 node spacings of degree 4.  y_bg: a
    background mass fraction of the heavy species (with none, the species'
    round-off far from the bubble reads as noise to the modal indicator).
    perturb: relative amplitude of smooth sine perturbations of the partial
    densities, the velocity and the pressure, so that no two neighbouring
    values are equal up to rounding (a tangent through minmod slopes is then
    defined by the data, not by rounding)."""
    sp = species_set([AIR, HEAVY], mu=mu)
    n_elem = nel[0] * nel[1] * nel[2]
    N = random_degrees(n_elem, 2, 6, seed)
    prob = make_problem([(nel, (0, 0, 0), (2, 1, 1))], sp, n_fv=7, N=N, riemann=riemann)
    rho2, p2, u2 = _post_shock(AIR["gamma"], SHOCK_MACH)
    T0 = 1.0 / (1.0 * sp["Rgas"][0])  # air at rho = p = 1
    width = 2 * (1.0 / nel[1]) / 5.0
    xs = 0.4

    def fn(x, y, z):
        r = np.sqrt((x - 0.8) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        Yb = y_bg + (1 - y_bg) * 0.5 * (1 - np.tanh((r - 0.2) / width))
        s = 0.5 * (1 - np.tanh((x - xs) / width))  # 1 behind the shock
        Rm = (1 - Yb) * sp["Rgas"][0] + Yb * sp["Rgas"][1]
        p = 1.0 + s * (p2 - 1.0)
        rho_pre = 1.0 / (Rm * T0)
        rho = rho_pre * (1 - s) + rho2 * s
        vx = s * u2
        if perturb:
            tw = 2 * np.pi
            g1 = np.sin(tw * (0.5 * x + 0.13)) * np.sin(tw * (y + 0.31)) * np.sin(tw * (z + 0.57))
            g2 = np.cos(tw * (0.5 * x + 0.71)) * np.sin(tw * (y + 0.17)) * np.cos(tw * (z + 0.43))
            g3 = np.sin(tw * (x + 0.29)) * np.cos(tw * (y + 0.61)) * np.sin(tw * (z + 0.11))
            p = p * (1 + perturb * g1)
            rho = rho * (1 + perturb * g2)
            return ([rho * (1 - Yb), rho * Yb],
                    (vx + perturb * g3, perturb * g1, perturb * g2), p)
        return [rho * (1 - Yb), rho * Yb], (vx, 0.0 * x, 0.0 * x), p

    return prob, build_state(prob, fn)


def _fourier_coeffs(rng, kmax, spectrum, solenoidal):
    k1 = np.arange(-kmax, kmax + 1)
    KX, KY, KZ = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    mask = (kk > 0) & (kk <= kmax)
    amp = np.where(mask, np.sqrt(spectrum(np.maximum(kk, 1e-12)) / (4 * np.pi * np.maximum(kk, 1) ** 2)), 0.0)
    ncomp = 3 if solenoidal else 1
    c = (rng.standard_normal((ncomp,) + kk.shape) + 1j * rng.standard_normal((ncomp,) + kk.shape)) * amp
    if solenoidal:
        kv = np.stack([KX, KY, KZ]).astype(float)
        kn = np.where(kk > 0, kk, 1.0)
        dot = (c * kv).sum(0) / kn ** 2
        c = c - dot[None] * kv
    return k1, c


def _eval_fourier(k1, c, X, Y, Z, L=2 * np.pi):
    """Real part of sum_k c_k exp(i 2pi/L k.x) at scattered points (small sets only)."""
    w = 2 * np.pi / L
    ex = np.exp(1j * w * np.asarray(X)[..., None] * k1)
    ey = np.exp(1j * w * np.asarray(Y)[..., None] * k1)
    ez = np.exp(1j * w * np.asarray(Z)[..., None] * k1)
    out = []
    for comp in c:
        t = np.einsum("pk,ijk->pij", ez.reshape(-1, len(k1)), comp, optimize=True)
        t = np.einsum("pj,pij->pi", ey.reshape(-1, len(k1)), t, optimize=True)
        out.append(np.real(np.einsum("pi,pi->p", ex.reshape(-1, len(k1)), t)).reshape(np.shape(X)))
    return out


def _fourier_on_mesh(prob, k1, c, L, chunk=4096):
    """Fourier series evaluated at the nodes of every DG element of a single
    structured domain, separably: the nodes of an element are a tensor grid,
    so the series is contracted axis by axis (z, then y, shared by all
    elements of a layer / row, then x per element).  Returns one flat array
    per component in the state's point layout (x fastest within an element)."""
    w = 2 * np.pi / L
    dims = prob["dims"][0]
    lo = prob["lo"][0]
    h = (prob["hi"][0] - lo) / dims
    _, pos, _, _ = element_index(prob)
    npd = points_per_dir(prob)
    off = np.zeros(len(npd) + 1, np.int64)
    off[1:] = np.cumsum(npd ** 3)
    out = [np.zeros(off[-1]) for _ in range(len(c))]
    for n in np.unique(npd):
        sel = np.nonzero(npd == n)[0]
        r = (dg_points(int(n), int(prob.get("nodes", 0))) + 1) / 2
        E = [np.exp(1j * w * ((np.arange(dims[a])[:, None] + r[None, :]) * h[a] + lo[a])[..., None] * k1)
             for a in range(3)]  # (n_a, n, K) per axis
        for q, comp in enumerate(c):
            T1 = np.einsum("ijk,zck->zijc", comp, E[2], optimize=True)       # (nz, K, K, n)
            T2 = np.einsum("ybj,zijc->yzibc", E[1], T1, optimize=True)       # (ny, nz, K, n, n)
            for s0 in range(0, len(sel), chunk):
                es = sel[s0:s0 + chunk]
                ix, iy, iz = pos[es, 0], pos[es, 1], pos[es, 2]
                v = np.einsum("eai,eibc->ecba", E[0][ix], T2[iy, iz], optimize=True)
                idx = off[es][:, None] + np.arange(int(n) ** 3)[None, :]
                out[q][idx.ravel()] = np.real(v).reshape(len(es), -1).ravel()
    return out


def turbulence(seed=0, nel=(48, 48, 48), riemann=0, mu=5e-4, Mt=0.3, k0=4.0, kmax=8, N0=None, y_bg=0.05, nodes=0,
               split=0):
    """Periodic [0,2pi]^3, 48^3 elements, N drawn from {1..7}, 3 species
    (gamma 1.4/1.3/1.67, M 29/44/4), N_FV = 8.  Random-phase solenoidal
    velocity with E(k) ~ k^4 exp(-2 (k/k0)^2), k0 = 4, scaled to turbulent Mach
    0.3; species blobs from thresholded Gaussian random fields smoothed by tanh
    over about 2 node spacings, on a background mass fraction y_bg of every
    species; p = 1 and uniform temperature."""
    sp = species_set([AIR, CO2, HELIUM], mu=mu)
    n_elem = nel[0] * nel[1] * nel[2]
    # N0 = None: degrees drawn from {1..7}; an integer: that degree everywhere
    N = random_degrees(n_elem, 1, 7, seed) if N0 is None else np.full(n_elem, N0, np.int8)
    L = 2 * np.pi
    prob = make_problem([(nel, (0, 0, 0), (L, L, L))], sp, n_fv=8, N=N, riemann=riemann, nodes=nodes, split=split)
    rng = np.random.default_rng(seed + 1)
    k1, cu = _fourier_coeffs(rng, kmax, lambda k: k ** 4 * np.exp(-2 * (k / k0) ** 2), True)
    kb, cb1 = _fourier_coeffs(rng, 3, lambda k: np.exp(-(k / 2.0) ** 2), False)
    _, cb2 = _fourier_coeffs(rng, 3, lambda k: np.exp(-(k / 2.0) ** 2), False)
    T0 = 1.0 / sp["Rgas"][0]
    c0 = math.sqrt(1.4)
    # normalise with a coarse sample: turbulent Mach number and blob field scales
    g = np.linspace(0, L, 24, endpoint=False)
    gx, gy, gz = (a.ravel() for a in np.meshgrid(g, g, g, indexing="ij"))
    vs = _eval_fourier(k1, cu, gx, gy, gz)
    vscale = Mt * c0 / math.sqrt(np.mean(vs[0] ** 2 + vs[1] ** 2 + vs[2] ** 2))
    s1 = _eval_fourier(kb, cb1, gx, gy, gz)[0].std()
    s2 = _eval_fourier(kb, cb2, gx, gy, gz)[0].std()
    width = 2 * (L / nel[0]) / 2.0  # 2 node spacings of the coarsest degree present (N = 1)
    vx, vy, vz = _fourier_on_mesh(prob, k1, cu, L)
    g1 = _fourier_on_mesh(prob, kb, cb1, L)[0] / s1
    g2 = _fourier_on_mesh(prob, kb, cb2, L)[0] / s2
    b1 = 0.5 * (1 + np.tanh(g1 / width))
    b2 = 0.5 * (1 + np.tanh(g2 / width))
    Y2 = y_bg + (0.6 - y_bg) * b1 * (1 - b2)
    Y3 = y_bg + (0.6 - y_bg) * b2
    Y1 = 1.0 - Y2 - Y3
    Rg = sp["Rgas"]
    rho = 1.0 / ((Y1 * Rg[0] + Y2 * Rg[1] + Y3 * Rg[2]) * T0)
    pts = dict(rk=[rho * Y1, rho * Y2, rho * Y3], v=[vscale * vx, vscale * vy, vscale * vz], p=np.ones_like(rho))
    return prob, _assemble(prob, pts)


def _assemble(prob, pts):
    """Conserved state from point fields in the state's point layout (rho E
    from the ideal-gas mixture relation of the initial condition)."""
    nk = len(prob["gamma"])
    cv = prob["Rgas"] / (prob["gamma"] - 1.0)
    cp = prob["gamma"] * cv
    rk, v, p = pts["rk"], pts["v"], pts["p"]
    rho = sum(rk)
    kap = sum(rk[k] * cp[k] for k in range(nk)) / sum(rk[k] * cv[k] for k in range(nk))
    fields = list(rk) + [rho * v[0], rho * v[1], rho * v[2],
                         p / (kap - 1.0) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)]
    npd = points_per_dir(prob)
    n3 = npd ** 3
    V = nk + 4
    poff = np.zeros(len(npd), np.int64)
    poff[1:] = np.cumsum(n3)[:-1]
    off, size = offsets(prob)
    U = np.empty(size)
    for n in np.unique(npd):
        es = np.nonzero(npd == n)[0]
        m3 = int(n) ** 3
        src = poff[es][:, None] + np.arange(m3)[None, :]
        blk = np.stack([f[src] for f in fields], axis=1)  # (ne, V, m3)
        dst = off[es][:, None] + np.arange(V * m3)[None, :]
        U[dst.ravel()] = blk.reshape(len(es), -1).ravel()
    return U


def mixing_layer(seed=0, nel=(16, 16, 16), N=4, delta=0.05, U0=0.5, amp=1e-2, mu=1e-3):
    """Temporal mixing layer for the adjoint: [0,1]^3 periodic, 16^3 elements,
    uniform N = 4, 3 species (air/CO2/helium).  A periodic pair of shear
    layers at y = 1/4 and 3/4 (tanh of thickness delta) carries v_x = +-U0 and
    the species: CO2 between the layers, air outside, 10 % helium everywhere;
    seeded random-phase velocity perturbations of amplitude amp; p = 1, uniform T."""
    sp = species_set([AIR, CO2, HELIUM], mu=mu)
    prob = make_problem([(nel, (0, 0, 0), (1, 1, 1))], sp, n_fv=N + 1, N=N)
    rng = np.random.default_rng(seed)
    ks = [(a, b, c) for a in range(1, 3) for b in range(1, 3) for c in range(0, 3)]
    ph = rng.uniform(0, 2 * np.pi, (3, len(ks)))
    T0 = 1.0 / sp["Rgas"][0]

    def fn(x, y, z):
        s = 0.5 * (np.tanh((y - 0.25) / delta) - np.tanh((y - 0.75) / delta))  # 1 between the layers
        pert = [amp * sum(np.sin(2 * np.pi * (a * x + b * y + c * z) + ph[q, m]) for m, (a, b, c) in enumerate(ks))
                / len(ks) for q in range(3)]
        Y2 = 0.8 * s + 0.05
        Y3 = 0.1 + 0 * x
        Y1 = 1.0 - Y2 - Y3
        Rm = Y1 * sp["Rgas"][0] + Y2 * sp["Rgas"][1] + Y3 * sp["Rgas"][2]
        rho = 1.0 / (Rm * T0)
        vx = U0 * (2 * s - 1) + pert[0]
        return [rho * Y1, rho * Y2, rho * Y3], (vx, pert[1], pert[2]), np.ones_like(x)

    return prob, build_state(prob, fn)


def batched_domains(seed=0, n_domains=256, mu=5e-4):
    """Many independent periodic domains in one context: n_d^3 elements with
    n_d drawn from {2..8} and one degree N_d from {1..7} per domain, 3 species,
    smooth random-phase states (unit boxes)."""
    rng = np.random.default_rng(seed)
    sp = species_set([AIR, CO2, HELIUM], mu=mu)
    doms, N = [], []
    for _ in range(n_domains):
        nd = int(rng.integers(2, 9))
        doms.append(((nd, nd, nd), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)))
        N += [int(rng.integers(1, 8))] * nd ** 3
    prob = make_problem(doms, sp, n_fv=8, N=np.array(N, np.int8))
    return prob, smooth_random_state(prob, seed, amp=0.05)


def domain_slices(prob):
    """Per domain: (problem of that domain alone, slice of the batched state)."""
    off, size = offsets(prob)
    out, e0 = [], 0
    for d, dm in enumerate(prob["dims"]):
        ne = int(np.prod(dm))
        sub = dict(prob, dims=prob["dims"][d:d + 1], lo=prob["lo"][d:d + 1], hi=prob["hi"][d:d + 1],
                   N=prob["N"][e0:e0 + ne].copy(), fv=prob["fv"][e0:e0 + ne].copy())
        end = off[e0 + ne] if e0 + ne < len(off) else size
        out.append((sub, slice(int(off[e0]), int(end))))
        e0 += ne
    return out


# Indicator thresholds {T_fv_on, T_fv_off, T_ref, T_crs} (configuration values).
THRESHOLDS = (2.0, 3.0, 3.5, 7.0)


# Supersonic Taylor-Green vortex (Sec. 4.3): Sutherland constant relative to the
# reference temperature (air: 110.4 K / 273.15 K), Prandtl number 0.71.
TGV_S_OVER_TREF = 110.4 / 273.15
TGV_THRESHOLDS = (2.0, 3.0, 3.0, 5.0)


def tgv(nel=32, N0=3, Ma=1.25, Re=1600.0, n_fv=9, nodes=0, riemann=0, fv=None):
    """Supersonic Taylor-Green vortex on [-pi, pi]^3 (Sec. 4.3): one gas with
    gamma = 1.4, rho_0 = 1, Ma_0 = sqrt(rho_0 / (gamma p_0)) = 1.25, Re_0 =
    rho_0 / mu_0 = 1600, isothermal start at T_0 = T_ref of Sutherland's law,
    v = (sin x cos y cos z, -cos x sin y cos z, 0),
    p = p_0 + rho_0/16 (cos 2x + cos 2y)(2 + cos 2z), rho = p / (R T_0).
    Elements start at degree N0 (a scalar or one per element) and FV flags fv;
    p-refinement on the pressure indicator, FV on the density indicator;
    N_FV = 9 as in the paper."""
    rho0 = 1.0
    p0 = rho0 / (1.4 * Ma * Ma)
    sp = species_set([AIR], mu=rho0 / Re, Pr=0.71)
    R = sp["Rgas"][0]
    T0 = p0 / (rho0 * R)
    L = np.pi
    prob = make_problem([((nel, nel, nel), (-L, -L, -L), (L, L, L))], sp, n_fv=n_fv, N=N0, fv=fv, riemann=riemann,
                        nodes=nodes)
    prob.update(sutherland=1, T_ref=T0, S_sutherland=TGV_S_OVER_TREF * T0, indicator_vars=1)

    def fn(x, y, z):
        p = p0 + rho0 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (2.0 + np.cos(2 * z))
        v = (np.sin(x) * np.cos(y) * np.cos(z), -np.cos(x) * np.sin(y) * np.cos(z), 0.0 * x)
        return [p / (R * T0)], v, p

    return prob, build_state(prob, fn)


def half_refined_wave(k=24, N_lo=2, N_hi=5, fv_frac=0.05, n_fv=8, seed=0, mu=1e-4, riemann=0):
    """Non-conforming mesh of Sec. 4.1 / 4.2 on the unit cube (Cartesian): the
    lower half in x at twice the resolution, (k, 2k, 2k) elements, the upper
    half (k/2, k, k), so both x interfaces carry type-3 mortars (Sec. 3.2.3);
    random degrees in [N_lo, N_hi] and FV elements (Sec. 4.1 draws both at
    random); 2 species; the density wave of Sec. 4.2 travelling along [1,1,1]."""
    sp = species_set([AIR, HELIUM], mu=mu)
    doms = chain_domains([(k, 2 * k, 2 * k, 0.5), (k // 2, k, k, 0.5)])
    ne = sum(int(np.prod(d[0])) for d in doms)
    prob = make_problem(doms, sp, n_fv=n_fv, N=random_degrees(ne, N_lo, N_hi, seed), fv=random_fv(ne, fv_frac, seed),
                        chain=1, riemann=riemann)

    def fn(x, y, z):
        s = 2 * np.pi * (x + y + z)
        rho = 1 + 0.2 * np.sin(s)
        Y = 0.5 + 0.2 * np.cos(s)
        return [rho * Y, rho * (1 - Y)], (0.5 + 0 * x, 0.5 + 0 * x, 0.5 + 0 * x), np.ones_like(x)

    return prob, build_state(prob, fn)


def shard_domains(prob, U, rank, world):
    """This rank's share of a batch of independent domains: domains taken in
    order of decreasing DOFs, each given to the rank with the fewest DOFs so far
    (ties to the lower rank).  Returns (problem of the share, its state, the
    domain ids, in increasing order)."""
    slices = domain_slices(prob)
    sizes = [sl.stop - sl.start for _, sl in slices]
    load = [0] * world
    owner = [0] * len(slices)
    for d in sorted(range(len(slices)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[d] = r
        load[r] += sizes[d]
    ids = [d for d in range(len(slices)) if owner[d] == rank]
    if not ids:
        return None, None, []
    subs = [slices[d][0] for d in ids]
    share = dict(prob, dims=np.concatenate([s["dims"] for s in subs]), lo=np.concatenate([s["lo"] for s in subs]),
                 hi=np.concatenate([s["hi"] for s in subs]), N=np.concatenate([s["N"] for s in subs]),
                 fv=np.concatenate([s["fv"] for s in subs]))
    Us = np.concatenate([U[slices[d][1]] for d in ids])
    return share, Us, ids
