"""The autotuner: host-side helpers (CPU) and a tuned run's parity (GPU)."""
import numpy as np
import pytest

from paper_1602_05856_gb300 import autotune, genomes


def test_prefix_sample_takes_the_same_prefix_of_every_string():
    seqs = [np.frombuffer(b"A" * n, np.uint8) for n in (1000, 3000, 50)]
    s = autotune.prefix_sample(seqs, 0.1, k=25)
    assert [x.size for x in s] == [135, 135, 50]  # 10% of 4050 bases, over 3 strings
    assert autotune._pow2_at_least(1) == 1 and autotune._pow2_at_least(1025) == 2048


def test_choice_options_reproduce_the_budgeted_workspace():
    """A choice's options size the workspace it was budgeted at, below the
    worst-case table reserve of the default options."""
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    m, n, k, bits, rounds = 10**7, 5, 25, 1 << 26, 2
    ws = autotune.full_workspace(m, n, k, bits, rounds, 4, 1 << 20, 300000)
    c = autotune.Choice(bits, 4, rounds, ws, 1.0, [], 1 << 20, 300000)
    assert T.twopaco_workspace_size(m, n, k, bits, rounds, c.options()) == ws
    assert ws < T.twopaco_workspace_size(m, n, k, bits, rounds, T.Options(hashes=4))
    assert c.options(hashes=6).hashes == 6
    c2 = autotune.Choice(bits, 4, rounds, ws, 1.0, [], 1 << 20, 300000, blocks_per_sm=2)
    assert c2.options().launch_blocks_per_sm == 2 and c.options().launch_blocks_per_sm == 0


@pytest.mark.gpu
def test_tuned_configuration_is_exact_and_fits_the_budget():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    seqs = genomes.named_set("plain_single", 0.1)
    k = 25
    choice = autotune.tune(seqs, k, bits_per_base=(4, 16), hashes=(3, 6), rounds=(1, 2),
                           sample_fraction=0.25, repeats=2, launch_shapes=(0, 2))
    assert choice.rounds == 1 and len(choice.trials) == 4
    assert set(choice.shape_ms) == {0, 2} and choice.blocks_per_sm in (0, 2)
    got, _ = T.twopaco_build_ex(seqs, k, choice.bits, choice.rounds, choice.options())
    want = O.junctions(genomes.concat(seqs), k)
    assert all(np.array_equal(g, w) for g, w in zip(got, want))
    # a budget one round cannot meet pushes the tuner to more rounds
    one_round = min(t.workspace for t in choice.trials if t.rounds == 1)
    tight = autotune.tune(seqs, k, budget_bytes=one_round - 1, bits_per_base=(4,), hashes=(4,),
                          rounds=(1, 4), sample_fraction=0.25, repeats=1)
    assert tight.rounds == 4 and tight.workspace < one_round
    with pytest.raises(ValueError):
        autotune.tune(seqs, k, budget_bytes=1024, bits_per_base=(4,), hashes=(4,), rounds=(1,),
                      sample_fraction=0.25, repeats=1)
