"""The kernels' bounded waits, made to run out on the GPU without a fault.

sl1m_selftest_bounded_wait runs a kernel whose threads wait on an mbarrier
that nobody arrives on (no copy is in flight, nothing is out of bounds).  The
wait must give up after its time limit on the GPU's global timer, set the
device fault flag and let the kernel end; the host must report SL1M_ERR_CUDA;
and the context must stay usable: its next calls succeed and a solve still
matches the FP64 oracle (Sect. 3 algorithm box)."""
import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_stays_usable(gpu_lib):
    ctx = gpu_lib.Context(0)
    for _ in range(2):                          # the flag is cleared and set again
        st, waited, limit = ctx.selftest_bounded_wait()
        assert st == gpu_lib.ERR_CUDA
        assert limit == 20_000_000
        assert limit <= waited <= limit + 20_000_000, waited
        assert "did not complete" in ctx.lib.sl1m_last_error(ctx.h).decode()
    w = synth.config1(scale=0.5)
    O = oracle.Problem(w.uvw, w.lm)
    V = oracle.forward(O, w.x_true) + w.noise
    P = ctx.problem()
    P.set_visibilities(w.uvw, V)
    P.set_pixels(w.lm)
    x = np.random.default_rng(1).random(w.n_pix)
    f = P.forward(x, gpu_lib.MIXED)              # succeeds: the flag was cleared
    assert np.max(np.abs(f - oracle.forward(O, x))) <= 1e-5 * np.max(np.abs(f))
    L, _ = oracle.power(O)
    lam = 0.02 * oracle.adjoint(O, V).max()
    img_o, _ = oracle.fista(O, V, lam, L, 30)
    for prec in (gpu_lib.FP64, gpu_lib.MIXED):
        img, stats = P.solve(lam, L=L, max_iter=30, precision=prec)
        assert np.max(np.abs(img - img_o)) <= 1e-4 * img_o.max()
    ctx.close()
