"""Open-output contractions on the GPU for the sampler: the 2^N_f
amplitudes over the open qubits against the FP64 oracle, for several
choices of the fixed bits on one cached tree."""
import numpy as np
import pytest

from oracle import tree
from paper_2002_01935_gb300 import inputs, planner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_01935_gb300 import build
    build.build()
    return _t


@pytest.mark.parametrize("mode", ["fp32", "tf32_split"])
def test_open_amplitudes_match_the_oracle(torch, mode):
    from paper_2002_01935_gb300 import sampling
    circ = inputs.random_circuit(3, 3, 6, seed=8)
    open_q = [8, 0, 4]
    prov = sampling.OpenAmplitudes(circ, open_q, mode=mode)
    fixed = prov.fixed
    rng = np.random.default_rng(2)
    try:
        for _ in range(3):
            x_u = [int(b) for b in rng.integers(0, 2, size=len(fixed))]
            got = prov(x_u)
            bits = [0] * 9
            for q, b in zip(fixed, x_u):
                bits[q] = b
            net = inputs.circuit_network(circ, bits, open_qubits=open_q)
            m, e = tree.contract_net(net, prov.pairs)
            ref = np.asarray(m) * 2.0 ** e
            assert got.shape == (2, 2, 2)
            assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
        s = sampling.sample(9, open_q, prov, 20, fidelity=0.5, seed=1)
        assert len(s) == 20 and all(len(b) == 9 for b, _ in s)
    finally:
        prov.close()
