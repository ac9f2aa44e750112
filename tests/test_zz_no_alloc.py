"""The allocation-free entry point (mlq_solve_noalloc), called through the C
ABI on CUDA tensors the test owns, against the regular mlq_solve on the same
inputs.  Callers that cannot allocate device memory when they need a solve (a
fixed-budget allocator owning the GPU's memory, a loop that must not take the
synchronisation an allocation may imply) use this call; its working memory is
a fixed static device array.

The file name makes pytest collect it last."""
import numpy as np
import pytest

from paper_2105_02007_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6   # the mixed-path tolerance of the parity tests


@pytest.fixture(scope="module")
def mlq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_02007_gb300 import build

    build.build()
    from paper_2105_02007_gb300 import mlq as m

    return m


def test_noalloc_matches_solve_twice_in_a_row(mlq):
    import torch

    m, K, S, dt, nsteps = 33, 8, 24, 0.05, 20
    modes, _ = mlq.build_kl(m, 0.09, 0.04, K)
    phi = mlq.centroid_table(m, modes, m)
    xi = inputs.gaussian_xi(7, 0, 0, S, K)
    with mlq.Context(0, mlq.MLQ_MIXED) as ctx:
        ctx.add_level(0, m, dt, nsteps)
        ctx.set_kl(0, phi)
        ref = ctx.solve(0, xi)
    assert np.all(ref["status"] == 0)

    dev = torch.device("cuda", 0)
    d_phi = torch.from_numpy(phi).to(dev)
    d_xi = torch.from_numpy(xi).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call in range(2):
        q = torch.full((S,), float("nan"), dtype=torch.float64, device=dev)
        st = torch.full((S,), -1, dtype=torch.int32, device=dev)
        it = torch.zeros(S, dtype=torch.int32, device=dev)
        mlq.solve_noalloc(m, dt, nsteps, d_phi, d_xi, q, status=st, iters=it, stream=stream)
        torch.cuda.synchronize(dev)
        qh = q.cpu().numpy()
        assert np.all(st.cpu().numpy() == 0), call
        assert np.all(it.cpu().numpy() > 0), call
        rel = np.max(np.abs(qh - ref["q_fine"]) / np.abs(ref["q_fine"]))
        assert rel < TOL_MIXED, (call, rel)


def test_noalloc_rejects_oversize_and_host_pointers(mlq):
    import torch

    dev = torch.device("cuda", 0)
    m, K = 257, 4
    S = 64                                  # ~0.5 GB of working memory: over the fixed scratch
    phi = torch.zeros((2 * (m - 1) ** 2, K), dtype=torch.float64, device=dev)
    xi = torch.zeros((S, K), dtype=torch.float64, device=dev)
    q = torch.zeros(S, dtype=torch.float64, device=dev)
    with pytest.raises(mlq.MLQError) as e:
        mlq.solve_noalloc(m, 0.01, 2, phi, xi, q)
    assert e.value.code == mlq.MLQ_ETOOBIG
    with pytest.raises(mlq.MLQError) as e:
        mlq.solve_noalloc(m, 0.01, 2, phi.cpu(), xi[:1], q[:1])
    assert e.value.code == -1


def test_noalloc_rejects_memory_of_another_gpu(mlq):
    import torch

    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU")
    m, K, S = 17, 4, 2
    phi = torch.zeros((2 * (m - 1) ** 2, K), dtype=torch.float64, device="cuda:1")
    xi = torch.zeros((S, K), dtype=torch.float64, device="cuda:0")
    q = torch.zeros(S, dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(0):
        with pytest.raises(mlq.MLQError) as e:
            mlq.solve_noalloc(m, 0.01, 2, phi, xi, q)
    assert e.value.code == -1
