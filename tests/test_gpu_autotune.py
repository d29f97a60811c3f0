"""The autotuner (ax_autotune, ax_batch_autotune) and per-instance latencies
of the batched solve, through the C ABI.

  - the chosen configuration is one of the candidates (FFT transform, or the
    tensor-core transform with a mode-solve kernel that covers nr), is read
    back by ax_get_option / ax_batch_config, and a mixed solve with it meets
    1e-8 in the oracle's FP64 true residual;
  - a second operator of the same shape takes the cached choice; with
    AX_TUNE_CACHE set, a new process reads the choice from the file;
  - per-instance latencies of a batched solve lie between 0 and the batch's
    wall time and differ between instances that converge at different
    iterations.
"""
import os
import subprocess
import sys
import tempfile
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_1002_3094_gb300 as P  # noqa: E402
from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs  # noqa: E402
from workloads import batched_instances, layered_inclusion_medium  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    return torch.device("cuda:0")


def _setup(nr, nz, dev, n_rhs=4, instance=3):
    med = layered_inclusion_medium(n_rhs=n_rhs, nominal_n=max(nr, nz), instance=instance)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(dev) for x in (kr, kz, q)], nr, nz)
    return op, O.Operator(kr, kz, q, O.Grid(nr, nz)), sample_rhs(med, nr, nz)


def _candidates(op):
    ids = [v for v in range(1, 15) if P.ax_set_option(op, "mode_kernel", v, raise_on_error=False) == P.AX_OK]
    P.ax_set_option(op, "mode_kernel", 0)
    return ids


@pytest.mark.parametrize("nr,nz", [(600, 200), (1024, 96), (300, 4100)])
def test_autotune_choice_and_solve(cuda, nr, nz):
    op, ora, f = _setup(nr, nz, cuda)
    ids = _candidates(op)
    assert P.ax_autotune(op, 4, 3) is None
    dst = int(P.ax_get_option(op, "dst_tensor"))
    mk = int(P.ax_get_option(op, "mode_kernel"))
    if nz > 4096:
        assert dst == 0
    assert dst in (0, 1) and (mk == 0 or mk in ids), (dst, mk, ids)
    fd = torch.from_numpy(f).to(cuda)
    u = torch.zeros_like(fd)
    st, _ = P.ax_solve(op, fd, u, 4, 1e-8, 5000, P.AX_PCG_MIXED)
    assert st == P.AX_OK
    un = u.cpu().numpy()
    for j in range(4):
        phi = ora.phi(f[j])
        assert np.linalg.norm(phi - ora.apply_A(un[j])) <= 1e-8 * np.linalg.norm(phi)
    # the same shape again: the cached choice, without timing
    op2, _, _ = _setup(nr, nz, cuda, instance=7)
    t0 = time.perf_counter()
    P.ax_autotune(op2, 4, 3)
    assert time.perf_counter() - t0 < 0.5
    assert (int(P.ax_get_option(op2, "dst_tensor")), int(P.ax_get_option(op2, "mode_kernel"))) == (dst, mk)
    with pytest.raises(P.AxError):
        P.ax_autotune(op2, 4, 0)
    P.ax_destroy_operator(op2)
    P.ax_destroy_operator(op)


def test_tune_cache_file_across_processes(cuda):
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import torch, paper_1002_3094_gb300 as P\n"
            "from paper_1002_3094_gb300.inputs import sample_operator_inputs\n"
            "from workloads import layered_inclusion_medium\n"
            "P.load_library()\n"
            "med = layered_inclusion_medium(n_rhs=2, nominal_n=640, instance=1)\n"
            "kr, kz, q = sample_operator_inputs(med, 640, 130)\n"
            "d = torch.device('cuda', 0)\n"
            "op = P.ax_setup_operator(*[torch.from_numpy(x).to(d) for x in (kr, kz, q)], 640, 130)\n"
            "P.ax_autotune(op, 2, 3)\n"
            "print(int(P.ax_get_option(op, 'dst_tensor')), int(P.ax_get_option(op, 'mode_kernel')))\n") % ROOT
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "tune.txt")
        env = dict(os.environ, AX_TUNE_CACHE=path)
        a = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        assert a.returncode == 0, a.stderr
        lines = open(path).read().split("\n")
        assert any("|640|130|0|2 " in ln for ln in lines), lines
        b = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        assert b.returncode == 0, b.stderr
        assert a.stdout.split() == b.stdout.split()


def test_batch_autotune_and_per_instance_latency(cuda):
    inst = [x for x in batched_instances(40) if x[0] * x[1] <= 511 * 511][:12]
    ops, fs, us, oras = [], [], [], []
    for nr, nz, med in inst:
        kr, kz, q = sample_operator_inputs(med, nr, nz)
        ops.append(P.ax_setup_operator(*[torch.from_numpy(x).to(cuda) for x in (kr, kz, q)], nr, nz))
        fs.append(torch.from_numpy(sample_rhs(med, nr, nz)[0]).to(cuda))
        us.append(torch.zeros((nr, nz), dtype=torch.float64, device=cuda))
        oras.append((O.Operator(kr, kz, q, O.Grid(nr, nz)), sample_rhs(med, nr, nz)[0]))
    b = P.ax_batch_create(ops)
    P.ax_batch_autotune(b, 2)
    lat0, groups = P.ax_batch_latency(b, len(ops))
    shapes = set()
    for g in range(groups):
        c = P.ax_batch_config(b, g)
        shapes.add((c["nr"], c["nz"]))
        assert c["dst_tensor"] in (0, 1) and c["members"] >= 1
    assert shapes == {(nr, nz) for nr, nz, _ in inst}
    with pytest.raises(P.AxError):
        P.ax_batch_config(b, groups)
    t0 = time.perf_counter()
    st, info = P.ax_batch_solve(b, fs, us, 1e-8, 20000, P.AX_PCG_MIXED)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3
    assert st == P.AX_OK
    lat, _ = P.ax_batch_latency(b, len(ops))
    assert all(0.0 < x <= wall + 1.0 for x in lat), (lat, wall)
    iters = [i["iters"] for i in info]
    if max(iters) >= min(iters) + 2 * 16:  # converged in different graph replays
        assert max(lat) > min(lat)
    for (ora, f), u in zip(oras, us):
        phi = ora.phi(f)
        assert np.linalg.norm(phi - ora.apply_A(u.cpu().numpy())) <= 1e-8 * np.linalg.norm(phi)
    P.ax_batch_destroy(b)
    for op in ops:
        P.ax_destroy_operator(op)
