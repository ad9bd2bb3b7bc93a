"""The 2M-oil gear bath of the bench, in the launch configuration bench.py
times (autotuned pair-pass variant): pair sets of a seeded sample of
particles checked bit-exact against the oracle's brute-force search over all
2.8M snapshot positions, plus pair symmetry on the sample."""
import numpy as np
import pytest

from paper_2512_09904_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_09904_b300 import build
    build.build()
    from paper_2512_09904_b300 import sph as S
    return S


def test_gear_bath_2m_sampled_pair_sets(sph, oracle):
    case = W.gear_bath(dx=1e-3, omega=600.0)
    ctx = sph.from_case(case, stream=0)
    ctx.sph_step(1)
    ctx.sph_autotune(steps_per_trial=1)
    ctx.sph_step(2)
    pos = ctx.sph_read_fields("pos")  # the snapshot of the next advection step
    ctx.sph_step(1)
    counts, lst = ctx.sph_read_neighbors()
    start = np.concatenate([[0], np.cumsum(counts)])
    n = case.n_total
    rng = np.random.default_rng(12)
    kind = W.flatten(case)["kind"]
    # oil, static walls and gear particles all represented
    idx = np.concatenate([rng.choice(np.nonzero(kind == 0)[0], 160, replace=False),
                          rng.choice(np.nonzero(kind != 0)[0], 96, replace=False)])
    R2 = case.support_radius() ** 2
    rc, rl = oracle.neighbors_of(pos, R2, idx, case.config["periodic_mask"], case.config["extent"])
    off = 0
    for q, i in enumerate(idx):
        got = lst[start[i]:start[i + 1]]
        ref = rl[off:off + rc[q]]
        off += rc[q]
        assert np.array_equal(got, ref), (int(i), len(got), len(ref))
        # symmetry: i is a partner of each of its partners
        for j in got[:8]:
            assert i in lst[start[j]:start[j + 1]]
    assert counts[idx].sum() == rc.sum() > 50 * len(idx)
    ctx.close()
