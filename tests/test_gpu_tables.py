"""The baked scattering table and its lookup against the oracle's quadrature.

IM(theta; beta) (Section 4: the a_F, a_B and forward spread of Eq. 6-9 are
formed from it) is compared element by element with the oracle's FP64
Gauss-Legendre integral on the whole 256 x 64 grid, in FP32 and in FP16, and
the shading code's bilinear lookup at off-grid points against the bilinear
interpolant of the oracle's grid values (the table read) and against the
oracle's integral at the point (the interpolation error of the grid).
"""
import math

import numpy as np
import pytest

import oracle
import paper_2405_10565_gb300 as hr

pytestmark = pytest.mark.gpu

BETA_LO, BETA_HI = 0.04, 0.68


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_10565_gb300.build import build
    build()
    c = hr.hr_create(0)
    yield c
    hr.hr_destroy(c)


def _grid(nt, nb):
    th = 0.5 * math.pi * np.arange(nt) / (nt - 1)
    be = BETA_LO + (BETA_HI - BETA_LO) * np.arange(nb) / (nb - 1)
    return th, be


@pytest.fixture(scope="module")
def oracle_grid(ctx):
    nt, nb = hr.hr_table_export(ctx)
    th, be = _grid(nt, nb)
    ref = np.array([[oracle.im(t, b) for t in th] for b in be])
    return nt, nb, ref


def test_table_elementwise_fp32_and_fp16(ctx, oracle_grid):
    nt, nb, ref = oracle_grid
    assert (nt, nb) == (256, 64)
    t32 = np.zeros((nb, nt), np.float32)
    t16 = np.zeros((nb, nt), np.uint16)
    hr.hr_table_export(ctx, t32, t16)
    e32 = np.abs(t32 - ref)
    h = t16.view(np.float16).astype(np.float64)
    e16 = np.abs(h / ref - 1)
    print(f"IM table: FP32 max abs error {e32.max():.2e}, FP16 max rel error {e16.max():.2e}, "
          f"values {ref.min():.3f}..{ref.max():.3f}")
    assert e32.max() <= 1e-6
    assert e16.max() <= 1e-3          # one FP16 rounding is 2^-11 = 4.9e-4 relative


@pytest.mark.parametrize("precision", [0, 1])
def test_lookup_off_grid(ctx, oracle_grid, precision):
    nt, nb, ref = oracle_grid
    th_g, be_g = _grid(nt, nb)
    rng = np.random.default_rng(5 + precision)
    m = 4000
    th = rng.uniform(0, 0.5 * math.pi, m).astype(np.float32)
    be = rng.uniform(BETA_LO, BETA_HI, m).astype(np.float32)
    # the grid's ends and a few points past them (clamped)
    th[:4] = [0.0, 0.5 * math.pi, -0.1, 2.0]
    be[:4] = [BETA_LO, BETA_HI, 0.02, 0.9]
    out = np.zeros(m, np.float32)
    hr.hr_im_lookup(ctx, th, be, out, precision)
    # bilinear interpolant of the oracle's grid values at the clamped point
    tc = np.clip(th.astype(np.float64), 0, 0.5 * math.pi)
    bc = np.clip(be.astype(np.float64), BETA_LO, BETA_HI)
    ft = tc / (0.5 * math.pi) * (nt - 1)
    fb = (bc - BETA_LO) / (BETA_HI - BETA_LO) * (nb - 1)
    it = np.minimum(ft.astype(int), nt - 2)
    ib = np.minimum(fb.astype(int), nb - 2)
    wt, wb = ft - it, fb - ib
    v = ((1 - wb) * ((1 - wt) * ref[ib, it] + wt * ref[ib, it + 1]) +
         wb * ((1 - wt) * ref[ib + 1, it] + wt * ref[ib + 1, it + 1]))
    err_abs = np.abs(out - v)
    err_rel = err_abs / v
    exact = np.array([oracle.im(float(a), float(b)) for a, b in zip(tc[:400], bc[:400])])
    err_grid = np.abs(v[:400] - exact)
    print(f"lookup precision {precision}: against the interpolant abs {err_abs.max():.2e} "
          f"rel {err_rel.max():.2e}; interpolant against the integral {err_grid.max():.2e}")
    if precision == 0:
        # table rounding (1e-6) and the FP32 weights' rounding times a cell's slope
        assert err_abs.max() <= 5e-6
    else:
        # one FP16 rounding (2^-11) of the values interpolated
        assert err_rel.max() <= 1e-3
    # Bilinear interpolation error of the grid, (h^2 / 8) max |f''| per axis, with
    # IM ~ 1 + cos(2 theta) exp(-8 beta^2): 2.0e-4 over beta (h = 0.0102,
    # |f''| <= 15.6) plus 1.9e-5 over theta (h = 0.0062, |f''| <= 4)
    assert err_grid.max() <= 2.5e-4
