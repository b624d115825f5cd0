"""GPU parity on the sine-wave stream of Sec. 5.1 (the paper's first experiment), shortened in time.

f(x) = sum_j c_j sin(pi j . x) on a 100 x 100 spatial grid with |j_k| <= 5 has exact spatial
ranks 2 f_k + 1 = 11 (closed form, Sec. 5.1). Halfway through the stream the time-mode frequency
bound grows from 5 to 7 (the rank bump of Table 1 / Fig. 3): the streaming rank must then grow on
the next slices. The CUDA path (through the C ABI) is compared with the FP64 oracle step by step
on the same seeded slices; bars as in test_gpu_parity.
"""

import numpy as np
import pytest

import oracle as O
from tests.test_gpu_parity import _compare_final, _run
from workloads import SineWave


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_16395_gb300 as p
    from paper_2308_16395_gb300 import build as b

    b.build()
    p.load_library()
    return p


@pytest.mark.gpu
@pytest.mark.parametrize("precision,dtype", [("fp64", "f64"), ("mixed", "f32")])
def test_sine_wave_rank_bump(pkg, precision, dtype):
    steps_each, n_init, tau = 60, 20, 1e-2
    sw = SineWave(n=(100, 100), steps_each=steps_each, freqs_a=(5, 5, 5), freqs_b=(5, 5, 7),
                  noise=1e-3)
    X = np.asfortranarray(np.stack([sw.slice(t) for t in range(sw.steps)], axis=-1))
    st, ts, Xs, recs = _run(pkg, X, n_init, tau, precision, dtype)
    # closed form: the spatial ranks stay 2 f_k + 1 = 11 at every step (the runner checks that
    # the library's ranks equal the oracle's at every step)
    for r in recs:
        assert r["ranks"][:2] == (11, 11), r
    # rank bump: the time-mode content gains 4 dimensions at t = steps_each; the streaming rank
    # grows on each of the first three slices after it
    rank_at = {r["t"]: r["ranks"][2] for r in recs}
    assert rank_at[steps_each] > rank_at[steps_each - 1]
    assert rank_at[steps_each + 2] - rank_at[steps_each - 1] >= 3
    _compare_final(pkg, st, ts, Xs, precision, "sine", recs)
    ts.close()


def test_sine_wave_oracle_bound_and_spatial_closed_form():
    """CPU pin of the same stream: the oracle alone keeps ranks (11, 11) and meets tau."""
    sw = SineWave(n=(100, 100), steps_each=30, freqs_a=(5, 5, 5), freqs_b=(5, 5, 7), noise=1e-3)
    X = np.asfortranarray(np.stack([sw.slice(t) for t in range(sw.steps)], axis=-1))
    st = O.init_stream(X[..., :15].copy(order="F"), 1e-2)
    for t in range(15, sw.steps):
        O.stream_update(st, X[..., t].copy(order="F"))
        assert st.ranks[:2] == (11, 11)
    Xh = O.reconstruct(st.C, st.Us)
    assert np.linalg.norm(X - Xh) <= 1e-2 * np.linalg.norm(X)
