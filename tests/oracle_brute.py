"""Independent brute-force restatements used to pin the oracle (tests only).

Nothing here calls the oracle's C code: random draws come from numpy's own
Philox4x64-10, resonance points from bisection on the comoving frequency,
cells from flooring the resonance position, optical depths from the
oscillator-strength form of the Sobolev optical depth."""
import numpy as np

C = 2.99792458e10
H = 6.62607015e-27
PI_E2_MC = np.pi * 4.80320471e-10 ** 2 / (9.1093837015e-28 * 2.99792458e10)


def philox_uniforms(seed, p, e):
    ctr = int(p) + (int(e) << 64)
    bg = np.random.Philox(counter=ctr - 1 if ctr > 0 else (1 << 256) - 1, key=int(seed))
    x = bg.random_raw(4).astype(np.uint64)
    return (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def largest_remainder(L, N):
    tot = 0.0
    for v in L:
        tot += v
    q = [(N * v) / tot for v in L]
    n = [int(np.floor(x)) for x in q]
    rem = sorted(range(len(L)), key=lambda c: (-(q[c] - n[c]), c))
    for k in range(N - sum(n)):
        n[rem[k]] += 1
    return np.concatenate([[0], np.cumsum(n)])


def tau_f_form(w, cell, line):
    """tau = (pi e^2 / m_e c) f lambda t (n_l - g_l n_u / g_u)."""
    lo, up = w.lo[line], w.up[line]
    nl, nu_ = w.pops[cell, lo], w.pops[cell, up]
    gl, gu = w.g_level[lo], w.g_level[up]
    return PI_E2_MC * w.f_lu[line] * w.lambda_A[line] * 1e-8 * w.t * (nl - gl * nu_ / gu)


def brute_packet(w, p, qoff, tau_min=1e-4, e_cut=1e-6):
    """Attenuation-mode history of packet p: list of (cell, line, value), fate,
    N_final.  Emission follows the documented draw layout."""
    R = w.v_max * w.t
    d = np.array([2 * R / w.nx, 2 * R / w.ny, 2 * R / w.nz])
    nn = np.array([w.nx, w.ny, w.nz])
    c = int(np.searchsorted(qoff, p, side="right") - 1)
    idx = np.array([c % w.nx, (c // w.nx) % w.ny, c // (w.nx * w.ny)])
    u = philox_uniforms(w.seed, p, 0)
    v = philox_uniforms(w.seed, p, 1)
    r0 = (-R + idx * d) + u[:3] * d
    mu = 2 * u[3] - 1
    ph = 2 * np.pi * v[0]
    st = np.sqrt(1 - mu * mu)
    n = np.array([st * np.cos(ph), st * np.sin(ph), mu])
    nu_lo, nu_hi = C / (w.band_A[1] * 1e-8), C / (w.band_A[0] * 1e-8)
    nu0 = nu_lo + v[1] * (nu_hi - nu_lo)
    ct = C * w.t
    nu_lab = nu0 / (1 - n @ r0 / ct)
    E0 = w.L_cell[c] / (qoff[c + 1] - qoff[c])
    N = E0 / (H * nu0)
    # exit distance from the cube (slab method)
    with np.errstate(divide="ignore"):
        t1 = (-R - r0) / n
        t2 = (R - r0) / n
    s_exit = np.min(np.maximum(t1, t2))
    nu_cmf = lambda s: nu_lab * (1 - n @ (r0 + s * n) / ct)
    lines_nu = C / (w.lambda_A * 1e-8)
    hits = []
    for l in range(w.nline):
        if not (lines_nu[l] <= nu0 and lines_nu[l] > nu_cmf(s_exit)):
            continue
        a, b = 0.0, s_exit
        for _ in range(200):
            m = 0.5 * (a + b)
            if nu_cmf(m) > lines_nu[l]:
                a = m
            else:
                b = m
        s = 0.5 * (a + b)
        cell_idx = np.floor((r0 + s * n + R) / d).astype(int)
        cell_idx = np.clip(cell_idx, 0, nn - 1)
        cell = int((cell_idx[2] * w.ny + cell_idx[1]) * w.nx + cell_idx[0])
        hits.append((s, -lines_nu[l], l, cell))
    hits.sort()
    out = []
    fate = 0
    for s, _, l, cell in hits:
        tau = tau_f_form(w, cell, l)
        if tau > tau_min:
            lo, up = w.lo[l], w.up[l]
            fcorr = 1 - w.g_level[lo] * w.pops[cell, up] / (w.g_level[up] * w.pops[cell, lo])
            dN = N * (-np.expm1(-tau))
            out.append((cell, l, dN / fcorr))
            N = N * np.exp(-tau)
            if N * H * lines_nu[l] < e_cut * E0:
                fate = 1
                break
    return out, fate, N, n, nu_lab
