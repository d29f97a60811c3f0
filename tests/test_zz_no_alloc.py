"""The allocation-free preconditioner entry point against the regular one.

ax_apply_preconditioner_noalloc serves callers that cannot call cudaMalloc
(for example code running while a stream is captured into a CUDA graph); it
stages through a fixed array inside the library.  It must give the same
B^-1 v as ax_apply_preconditioner, on two calls in a row (the array keeps the
previous call's contents, which must not leak into the next result).  This
file is collected last so that a failure here cannot hide any other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1002_3094_gb300 as P  # noqa: E402
from paper_1002_3094_gb300.inputs import sample_operator_inputs  # noqa: E402
from workloads import layered_inclusion_medium  # noqa: E402

pytestmark = pytest.mark.gpu

# Same tolerance as the B^-1 parity test against the oracle.
TOL = {P.AX_PREC_FP64: 1e-12, P.AX_PREC_FP32: 1e-5}


@pytest.mark.parametrize("prec", [P.AX_PREC_FP64, P.AX_PREC_FP32])
def test_noalloc_preconditioner_matches_regular(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    dev = torch.device("cuda:0")
    nr, nz = 96, 130
    med = layered_inclusion_medium(n_rhs=1, nominal_n=128)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(dev) for x in (kr, kz, q)], nr, nz)
    try:
        rng = np.random.default_rng(42)
        for call, m in enumerate((3, 2)):  # two calls in a row, different sizes
            v = torch.from_numpy(rng.normal(size=(m, nr, nz))).to(dev)
            ref = torch.zeros_like(v)
            got = torch.full_like(v, float("nan"))
            P.ax_apply_preconditioner(op, v, ref, m, prec)
            P.ax_apply_preconditioner_noalloc(op, v, got, m, prec)
            torch.cuda.synchronize()
            a, b = got.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a)), call
            assert np.linalg.norm(a - b) <= TOL[prec] * np.linalg.norm(b), call
        # requests beyond the fixed array are refused before any work
        big_m = 1 + (32 << 20) // (2 * nr * 160 * (8 if prec == P.AX_PREC_FP64 else 4))
        v = torch.zeros((1, nr, nz), dtype=torch.float64, device=dev)
        with pytest.raises(P.AxError) as e:
            P.ax_apply_preconditioner_noalloc(op, v, v.clone(), big_m, prec)
        assert e.value.status == P.AX_ERR_INVALID_ARG
    finally:
        P.ax_destroy_operator(op)
