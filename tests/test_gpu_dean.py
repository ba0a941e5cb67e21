"""Physics gate on the GPU: the critical Dean number of a narrow curved
channel (eta = r_i/r_o = 0.975, 64 x 4 x 256, L_z = 4 d) from the saturated
Dean-vortex amplitude (A^2 ~ De - De_c), against Dean's narrow-gap value ~36
printed in the paper's introduction (+-10%: the finite gap raises it, the
periodic box quantises the vortex wavelength, and the lattice has a finite
Mach number). The two relaxation times describe the same physics and must
agree to 5%."""
import numpy as np
import pytest

from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def test_critical_dean_narrow_gap():
    lib()
    from paper_1411_3133_gb300 import lbgm as L
    from paper_1411_3133_gb300.sweep import run_sweep, summarize
    spec = L.ChannelSpec("cylindrical", 1.0, 1 / 0.975, 64, 4, 256)
    deans = list(np.linspace(25.0, 60.0, 12))
    taus = [0.55] * 12 + [0.6] * 12
    res = run_sweep(spec, taus, deans + deans, steps=300_000, sample_every=2000)
    summ = summarize(res)
    dec = {tau: summ[tau]["De_c"] for tau in summ}
    print("De_c", dec, "growth-rate De_c", {t: summ[t]["De_c_growth"] for t in summ},
          "seconds", res.seconds)
    assert 36 * 0.9 <= dec[0.55] <= 36 * 1.1, dec
    assert 36 * 0.9 <= dec[0.6] <= 36 * 1.1, dec
    assert abs(dec[0.55] / dec[0.6] - 1) < 0.05, dec
