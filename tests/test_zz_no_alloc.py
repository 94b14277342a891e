"""The allocation-free solve, bfmri_pcg_solve_static, against bfmri_sample_W (needs a GB300).

Some callers cannot allocate device memory while they run: code inside another framework's
memory pool, a process whose device footprint is fixed after start-up, or a real-time loop
that cannot afford the device synchronisation that cudaMalloc/cudaFree imply. For them the
library offers one solve whose scratch lives in a static device array. This test hands it
the exact system that bfmri_sample_W solves (same blocks, same perturbed right-hand side,
same start value) and checks that both give the same draw, within the draw tolerance of the
other GPU tests (1e-8 relative L2), on two calls in a row (the second call must not see the
first call's leftovers). This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1606_00980_gb300 import synth

pytestmark = pytest.mark.gpu

SEED = 4321


def neighbour_planes(mask, neighbourhood, ld):
    """[6][ld] int32: compact index of the -x,+x,-y,+y,-z,+z in-mask neighbour, or -1."""
    nz, ny, nx = mask.shape
    flat = mask.reshape(-1) != 0
    lin = np.flatnonzero(flat)
    index_of = np.full(flat.size, -1, dtype=np.int64)
    index_of[lin] = np.arange(len(lin))
    x, y, z = lin % nx, (lin // nx) % ny, lin // (nx * ny)
    out = np.full((6, ld), -1, dtype=np.int32)
    steps = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    for d, (dx, dy, dz) in enumerate(steps[:neighbourhood]):
        xx, yy, zz = x + dx, y + dy, z + dz
        ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        idx = np.full(len(lin), -1, dtype=np.int64)
        idx[ok] = index_of[((zz * ny + yy) * nx + xx)[ok]]
        out[d, :len(lin)] = idx
    return out


def packed_planes(blocks, ld):
    N, D, _ = blocks.shape
    out = np.zeros((D * (D + 1) // 2, ld))
    for i in range(D):
        for j in range(i + 1):
            out[i * (i + 1) // 2 + j, :N] = blocks[:, i, j]
    return out


def padded(v, ld):
    out = np.zeros((v.shape[0], ld))
    out[:, :v.shape[1]] = v
    return out


def compare_twice(w, state_seed):
    """Hands bfmri_pcg_solve_static the system bfmri_sample_W solves for two draw counters in
    a row and checks the solutions agree (1e-8 relative L2); neither call may take device
    memory from PyTorch's allocator, and the second call (its kernels already loaded) may not
    lower the device's free memory either."""
    import torch

    from paper_1606_00980_gb300 import bfmri
    from paper_1606_00980_gb300.bfmri import Model

    m = Model.from_workload(w, delta=1e-12, seed=SEED)
    m.precompute_stats()
    rng = np.random.default_rng(state_seed)
    m.set_state(W=w.W_true + 0.1 * rng.standard_normal(w.W_true.shape), A=w.A_true,
                lam=rng.uniform(0.5, 2.0, w.N), alpha=rng.uniform(0.3, 3.0, w.K),
                beta=rng.uniform(2.0, 9.0, w.P))
    N, D = w.N, w.K
    ld = (N + 31) // 32 * 32
    lib = bfmri.load_library()
    assert lib.bfmri_pcg_static_bytes(ld, D) <= lib.bfmri_pcg_static_capacity()
    dev = torch.device("cuda")
    nbr = torch.from_numpy(neighbour_planes(w.mask, w.neighbourhood, ld)).to(dev)
    stream = torch.cuda.current_stream()
    for call, counter in enumerate((3, 4)):
        x0 = m.get_state()["W"]
        blocks, _, bpert = m.build_system(0, counter)
        alpha = m.get_state()["alpha"]
        W_ref, info_ref = m.sample_W(counter)          # the existing entry point
        Bp = torch.from_numpy(packed_planes(blocks, ld)).to(dev)
        sc = torch.from_numpy(alpha.copy()).to(dev)
        b = torch.from_numpy(padded(bpert, ld)).to(dev)
        x = torch.from_numpy(padded(x0, ld)).to(dev)
        torch.cuda.synchronize()
        torch_before = torch.cuda.memory_allocated()
        free_before = torch.cuda.mem_get_info()[0]
        info = bfmri.bfmri_pcg_solve_static(N, D, w.neighbourhood, nbr.data_ptr(), ld,
                                            Bp.data_ptr(), sc.data_ptr(), b.data_ptr(),
                                            x.data_ptr(), 1e-12, 3000, stream.cuda_stream)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == torch_before
        if call == 1:
            assert torch.cuda.mem_get_info()[0] >= free_before
        got = x.cpu().numpy()[:, :N]
        assert info.rel_residual <= 1e-12
        err = np.linalg.norm(got - W_ref) / np.linalg.norm(W_ref)
        assert err <= 1e-8, f"call with counter {counter}: rel L2 {err:.2e}"
    m.close()


def test_static_solve_matches_sample_W_twice():
    """About 600 voxels: the resident solver (one CTA per SM holds all of them)."""
    compare_twice(synth.small3d(seed=21, dims=(12, 10, 7), K=5, P=2, T=50), 2)


def test_static_solve_matches_sample_W_twice_streaming():
    """About 65k voxels at D = 6, near the 32 MiB limit: more voxels than the resident solver
    holds, so the streaming solver runs with its work vectors and partial-sum rows carved out
    of the static array."""
    w = synth.request_workload(seed=22, N_target=65000, K=6, T=40, P=1)
    assert 152 * 384 < w.N
    compare_twice(w, 3)


def test_static_solve_rejects_a_leading_dimension_not_a_multiple_of_32():
    from paper_1606_00980_gb300 import bfmri
    with pytest.raises(bfmri.BfmriError) as ei:
        bfmri.bfmri_pcg_solve_static(100, 3, 6, 1, 101, 1, 1, 1, 1, 1e-8, 10)
    assert ei.value.status == -1 and "multiple of 32" in str(ei.value)


def test_static_solve_rejects_oversized_problems():
    from paper_1606_00980_gb300 import bfmri
    lib = bfmri.load_library()
    ld = 10_000_000 // 32 * 32
    assert lib.bfmri_pcg_static_bytes(ld, 12) > lib.bfmri_pcg_static_capacity()
    with pytest.raises(bfmri.BfmriError) as ei:
        bfmri.bfmri_pcg_solve_static(ld, 12, 6, 1, ld, 1, 1, 1, 1, 1e-8, 10)
    assert ei.value.status == -1 and "static area" in str(ei.value)
