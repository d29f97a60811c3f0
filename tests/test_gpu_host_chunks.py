"""Host-buffer solves (AX_FLAG_HOST_BUFFERS) in right-hand-side chunks whose
copies overlap the solve (option host_chunks), through the C ABI.

Every right-hand side iterates on its own with fixed-order reductions, so a
chunked solve must give the device-buffer solve's answer bit for bit, with the
same iteration counts, also with an initial guess, uneven last chunks and
host_chunks = 1 (no chunking)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1002_3094_gb300 as P  # noqa: E402
from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs  # noqa: E402
from workloads import layered_inclusion_medium  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    return torch.device("cuda:0")


@pytest.mark.parametrize("m,chunks", [(8, 4), (11, 4), (9, 2), (6, 1)])
@pytest.mark.parametrize("method", [P.AX_PCG_MIXED, P.AX_PCG_FP64])
def test_chunked_host_solve_equals_device_solve(cuda, m, chunks, method):
    nr, nz = 160, 130
    med = layered_inclusion_medium(n_rhs=m, nominal_n=160, instance=5)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(cuda) for x in (kr, kz, q)], nr, nz)
    P.ax_set_option(op, "host_chunks", chunks)
    assert P.ax_get_option(op, "host_chunks") == chunks
    f = sample_rhs(med, nr, nz)
    fd = torch.from_numpy(f).to(cuda)
    ud = torch.zeros_like(fd)
    st, idev = P.ax_solve(op, fd, ud, m, 1e-8, 5000, method)
    assert st == P.AX_OK
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.zeros_like(fh).pin_memory()
    st, ihost = P.ax_solve(op, fh, uh, m, 1e-8, 5000, method, P.AX_FLAG_HOST_BUFFERS)
    assert st == P.AX_OK
    assert np.array_equal(uh.numpy(), ud.cpu().numpy())
    assert [i["iters"] for i in ihost] == [i["iters"] for i in idev]
    # with a guess (half the solution), kept by the gate
    g = (0.5 * ud).cpu()
    ud2 = (0.5 * ud).clone()
    flags = P.AX_FLAG_USE_GUESS | P.AX_FLAG_CHECK_GUESS
    st, i2 = P.ax_solve(op, fd, ud2, m, 1e-8, 5000, method, flags)
    assert st == P.AX_OK
    uh2 = g.pin_memory()
    st, i3 = P.ax_solve(op, fh, uh2, m, 1e-8, 5000, method, flags | P.AX_FLAG_HOST_BUFFERS)
    assert st == P.AX_OK
    assert np.array_equal(uh2.numpy(), ud2.cpu().numpy())
    assert [i["guess_accepted"] for i in i3] == [i["guess_accepted"] for i in i2]
    with pytest.raises(P.AxError):
        P.ax_set_option(op, "host_chunks", 0)
    P.ax_destroy_operator(op)
