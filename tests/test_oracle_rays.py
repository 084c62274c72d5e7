"""Pins of the oracle's RAYS sampler (Sec. 2.3: from the middle of every
cell, one ray per wavelength bin and viewer) against things other than
itself (no GPU).

- The ray count of the paper's validation pass (golden fixture): 17,100
  zones x the 0.1 % bins of 400-15000 A x 400 viewers = 2.5e10 rays.
- Optically thin: every ray escapes into its own viewer with its emission
  share, so the energy per viewer is the emission times dOmega_k / 4 pi
  exactly, and in total the emission.
- A single emission line, optically thin: every ray's lab wavelength follows
  from its cell centre and viewer direction by the first-order Doppler
  formula; the spectrum binned from that restatement equals the oracle's.
"""
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
C = 2.99792458e10


def _golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_ray_count.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_ray_count_of_the_paper_pass():
    g = _golden()
    # 38 x 15 x 30 cells, every one emitting, band 400-15000 A on the 0.1 % grid from 400 A
    w = synth.uniform_sphere(n=2, n_packets=1, n_lines=3, seed=1)
    w.nx, w.ny, w.nz = 38, 15, 30
    nc = w.nx * w.ny * w.nz
    assert nc == g["zones"]
    w.L_cell = np.ones(nc)
    for k in ("rho", "Te", "ne", "deposition"):
        setattr(w, k, np.ones(nc))
    w.n_ion_density = np.ones((nc, 1))
    w.pops = np.ones((nc, w.nlev))
    w.band_A = (g["lambda_lo_A"], g["lambda_hi_A"])
    w.lambda_A = np.array([500.0, 1000.0, 5000.0])
    nb = int(np.ceil(np.log(g["lambda_hi_A"] / g["lambda_lo_A"]) / np.log1p(g["dlog"]))) + 5
    w.spec_band_A = (g["lambda_lo_A"], nb)
    n = oracle.ray_count(w, n_theta=20, n_phi=20, spec_dlog=g["dlog"])
    bins = n // (nc * 400)
    assert n == nc * 400 * bins
    # the bins overlapping 400-15000 A: 3626 whole ones and the partial last one
    assert bins == int(np.floor(np.log(g["lambda_hi_A"] / g["lambda_lo_A"]) / np.log1p(g["dlog"]))) + 1
    assert n == pytest.approx(g["rays"], rel=0.01)


def _thin(w, emission="band"):
    w.pops = w.pops * 1e-30
    return w


@pytest.mark.parametrize("views", [(9, 10), (20, 20)])
def test_thin_rays_carry_the_emission_isotropically(views):
    nt, nph = views
    w = _thin(synth.uniform_sphere(n=6, n_packets=1, seed=5))
    o = oracle.transport(w, sampler="rays", n_theta=nt, n_phi=nph, spec_dlog=0.01, per_packet=True)
    L = o["ledger"]
    assert L["events"] == 0
    assert L["emit_E"] == pytest.approx(w.L_cell.sum(), rel=1e-9)      # (a sum over ~1e6 rays)
    assert L["esc_E"] == pytest.approx(L["emit_E"], rel=0.02)          # lab frame: Doppler factors
    # comoving energy per viewer: N h nu_0 summed over the rays of each viewer
    pk = o["pkt"]
    Ecmf = pk[:, 8] * 6.62607015e-27 * pk[:, 9]
    k = np.arange(o["n"]) % (nt * nph)
    per_view = np.bincount(k, weights=Ecmf, minlength=nt * nph)
    th = np.linspace(0.0, np.pi, nt + 1)
    dOm = np.repeat(2 * np.pi / nph * (np.cos(th[:-1]) - np.cos(th[1:])), nph)
    np.testing.assert_allclose(per_view, w.L_cell.sum() * dOm / (4 * np.pi), rtol=1e-10)
    # every ray escapes towards its own viewer
    assert np.array_equal(pk[:, 4], k.astype(float))


def test_single_line_rays_doppler_restatement():
    w = _thin(synth.single_line_sphere(n=6, n_packets=1, seed=7, lam_A=6000.0))
    nt, nph, dlog = 7, 10, 2e-4
    lam0 = 6000.0 * (1 - 0.03)
    nb = int(np.log(1.06 / 0.97) / np.log1p(dlog)) + 1
    w.spec_band_A = (lam0, nb)
    o = oracle.transport(w, sampler="rays", emission="lines", n_theta=nt, n_phi=nph,
                         spec_dlog=dlog, per_packet=True)
    R = w.v_max * w.t
    d = 2 * R / w.nx
    nu_l = C / (6000.0 * 1e-8)
    spec = np.zeros((nt * nph, nb))
    Lc, _ = oracle.emission(w, n_packets=1, emission="lines")
    cells = np.nonzero(Lc > 0)[0]
    th = np.linspace(0.0, np.pi, nt + 1)
    w_k = np.repeat(2 * np.pi / nph * (np.cos(th[:-1]) - np.cos(th[1:])), nph) / (4 * np.pi)
    for c in cells:
        idx = np.array([c % w.nx, (c // w.nx) % w.ny, c // (w.nx * w.ny)])
        r = -R + (idx + 0.5) * d
        for it in range(nt):
            for ip in range(nph):
                k = it * nph + ip
                tc, pc = np.pi * (it + 0.5) / nt, 2 * np.pi * (ip + 0.5) / nph
                n = np.array([np.sin(tc) * np.cos(pc), np.sin(tc) * np.sin(pc), np.cos(tc)])
                nu_lab = nu_l / (1 - n @ r / (C * w.t))
                lam = C / nu_lab * 1e8
                b = int(np.floor(np.log(lam / lam0) / np.log1p(dlog)))
                E0 = Lc[c] * w_k[k]
                spec[k, b] += E0 * nu_lab / nu_l                # lab energy of N = E0 / (h nu_l)
    m = spec > 0
    assert np.array_equal(m, o["spec"] > 0)
    np.testing.assert_allclose(o["spec"][m], spec[m], rtol=1e-12)
