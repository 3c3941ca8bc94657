"""The allocation-free headspace mean, for callers that cannot allocate
device memory (fixed device budgets, real-time coupling loops, foreign
allocators), against the reduction that chad_step performs.

Collected last on purpose: it uses the library's static scratch array and
must pass in a fresh process as well as after every other test.

Reference: run one interval with a per-particle headspace (no averaging) and
one with a shared headspace from the same state; within an interval the
particles evolve independently, so the shared run's gas states are the
per-digester means of the per-particle run's.
"""
import numpy as np
import pytest

from paper_2311_08927_gb300 import chad as CH
from paper_2311_08927_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_08927_gb300 import build
    build.build()
    CH.lib()


def _one_interval(pop, headspace):
    sim = CH.Simulator(pop, headspace=headspace, fixed_substeps=2)
    sim.load()
    sim.step(60.0, 1)
    out = sim.read()
    sim.close()
    return out["y"]


def _case(n, seed):
    pop = I.config_population(5, n=n, seed_offset=seed)
    y_free = _one_interval(pop, CH.HEADSPACE_PARTICLE)
    y_shared = _one_interval(pop, CH.HEADSPACE_SHARED)
    return pop, y_free, y_shared


def test_noalloc_mean_matches_chad_step_reduction_twice():
    import torch
    L = CH.lib()
    stream = torch.cuda.Stream()
    for seed, n in ((0, 9000), (1, 20000)):  # two calls in a row, different inputs
        pop, y_free, y_shared = _case(n, seed)
        off = np.ascontiguousarray(pop.offsets, dtype=np.int64)
        nd = len(pop.digesters)
        y_dev = torch.from_numpy(np.ascontiguousarray(y_free)).cuda()
        mean = torch.full((nd, 3), float("nan"), dtype=torch.float64, device="cuda")
        # the copy and the fill above are queued on torch's current stream;
        # the call runs on another stream, which must wait for them
        stream.wait_stream(torch.cuda.current_stream())
        code = L.chad_headspace_mean_noalloc(y_dev.data_ptr(), y_dev.shape[1], nd,
                                             off.ctypes.data, mean.data_ptr(),
                                             stream.cuda_stream)
        assert code == 0
        stream.synchronize()
        m = mean.cpu().numpy()
        for d in range(nd):
            a, b = off[d], off[d + 1]
            if b == a:
                continue
            ref = y_shared[26:29, a]
            assert np.all(y_shared[26:29, a:b] == ref[:, None])
            # same chunks, same fixed trees, same division: bit-identical
            assert np.array_equal(m[d], ref), (d, m[d], ref)


def test_noalloc_rejects_sizes_beyond_its_limits():
    L = CH.lib()
    y = np.zeros(1)
    mean = np.zeros(3)
    too_many = np.arange(1026, dtype=np.int64)  # 1025 digesters
    assert L.chad_headspace_mean_noalloc(y.ctypes.data, 2000, 1025, too_many.ctypes.data,
                                         mean.ctypes.data, None) == 1
    huge = np.array([0, 16385 * 4096], dtype=np.int64)  # 16385 chunks
    assert L.chad_headspace_mean_noalloc(y.ctypes.data, 16385 * 4096, 1, huge.ctypes.data,
                                         mean.ctypes.data, None) == 1
    bad = np.array([0, 10, 5], dtype=np.int64)
    assert L.chad_headspace_mean_noalloc(y.ctypes.data, 10, 2, bad.ctypes.data,
                                         mean.ctypes.data, None) == 1
