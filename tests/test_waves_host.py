"""Host-only: the memory-budgeted waves of a batch (paper_2506_17626_gb300.waves).
Every workspace size is the library's rfm_problem_size; no GPU needed."""
import pytest

import synth


@pytest.fixture(scope="module")
def W():
    from paper_2506_17626_gb300 import build
    build.build()
    from paper_2506_17626_gb300 import waves
    return waves


def test_waves_cover_the_batch_in_order_within_the_budget(W):
    probs = [synth.batched_instance(i, p_range=(20, 40)) for i in range(24)]
    sizes = [W.workspace_bytes([p]) for p in probs]
    budget = int(2.5 * max(sizes))
    waves = W.plan_waves(probs, budget)
    assert [i for w in waves for i in w] == list(range(len(probs)))
    for w in waves:
        assert W.workspace_bytes([probs[i] for i in w]) <= budget
    # greedy: the next instance would not have fitted into the previous wave
    for w, nxt in zip(waves, waves[1:]):
        assert W.workspace_bytes([probs[i] for i in w + [nxt[0]]]) > budget
    # a system's workspace is at least the sum of its instances' arenas less the shared records
    assert W.workspace_bytes(probs[:3]) >= 0.9 * sum(sizes[:3])


def test_waves_respect_the_instance_limit_and_reject_oversized_instances(W):
    probs = [synth.poisson1d(S=4, K=8, n=40, seed=i) for i in range(70)]
    waves = W.plan_waves(probs, 1 << 40)
    assert [len(w) for w in waves] == [64, 6]
    with pytest.raises(ValueError):
        W.plan_waves([synth.poisson2d(S=6, K=50, n=60)], 1024)
