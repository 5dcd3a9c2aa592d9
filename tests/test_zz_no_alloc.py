"""The allocation-free far-field entry point gives the same RCS as the allocating one.

Some callers cannot allocate device memory at the moment they ask for the RCS (their device memory
is held by another framework's pool, or they run in a loop that must not allocate).
swm_far_field_noalloc serves them from a fixed scratch array compiled into the library.  This file
is named to be collected last, so a run that stops at the first failure has already run every
other test.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

K = 2.0 * math.pi


def _case(seed, nw, n_rhs, n_obs):
    import torch

    from synth import cloud_uniform_cube

    cl = cloud_uniform_cube(nw, 6.0, seed=seed)
    rng = np.random.default_rng(seed)
    m = cl.nseg.astype(np.int64) - 1
    off = np.concatenate([[0], np.cumsum(m)])
    cur = rng.standard_normal((n_rhs, off[-1])) + 1j * rng.standard_normal((n_rhs, off[-1]))
    obs = np.stack([rng.uniform(0, math.pi, n_obs), rng.uniform(0, 2 * math.pi, n_obs)], 1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return [t(cl.centres), t(cl.dirs), t(cl.lengths), t(cl.nseg), t(off), K, t(cur), t(obs)]


def test_noalloc_matches_allocating_entry_point_on_two_calls_in_a_row():
    import torch

    from paper_2410_03060_gb300 import swm

    # the second call is smaller, so stale partial sums of the first could only leak in if the
    # shared scratch were read before being written
    for seed, nw, n_rhs, n_obs in ((1, 300, 3, 97), (2, 120, 2, 41)):
        args = _case(seed, nw, n_rhs, n_obs)
        ref = torch.zeros((n_rhs, n_obs, 2), dtype=torch.float64, device="cuda")
        got = torch.zeros_like(ref)
        swm.swm_far_field(None, *args, ref)
        swm.swm_far_field_noalloc(None, *args, got)
        torch.cuda.synchronize()
        ref, got = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) / np.max(ref) < 1e-10


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch

    from paper_2410_03060_gb300 import swm

    args = _case(3, 20, 2, 90_000)  # 180,000 incidence-observation pairs > 174,762
    out = torch.zeros((2, 90_000, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(swm.SwmError) as e:
        swm.swm_far_field_noalloc(None, *args, out)
    assert "scratch" in str(e.value)
