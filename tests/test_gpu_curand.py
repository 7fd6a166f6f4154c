"""The oracle's Philox4x32-10 against cuRAND's device-API generator (an
independent implementation): curand_init(seed, subsequence, offset) with
subsequence = t_index + 2^32 stream and offset = 4 (q + 2^32 n) starts at the
128-bit counter (q, n, t_index, stream) under key (seed low, seed high), so
its first curand4() block must equal the oracle's Philox block there -- the
counter layout of the parameter sampler."""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_tool(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("curand") / "curand_philox")
    subprocess.run([nvcc, "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                    os.path.join(HERE, "native", "curand_philox.cu")], check=True, timeout=300)
    return exe


def test_philox_against_curand(orc, curand_tool):
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(500):
        seed = int(rng.integers(0, 2 ** 63))
        q, n = int(rng.integers(0, 2 ** 20)), int(rng.integers(0, 2 ** 30))   # 4 (q + 2^32 n) < 2^64
        t, stream = int(rng.integers(0, 2 ** 32)), int(rng.integers(0, 4))
        cases.append((seed, q, n, t, stream))
    cases += [(0, 0, 0, 0, 0), (2 ** 64 - 1, 2 ** 32 - 1, 2 ** 30 - 1, 2 ** 32 - 1, 2 ** 31)]
    lines = "".join("%d %d %d\n" % (s, t + (st << 32), 4 * (q + (n << 32))) for s, q, n, t, st in cases)
    out = subprocess.run([curand_tool], input=lines, capture_output=True, text=True, check=True, timeout=120).stdout
    got = np.array([[int(v) for v in l.split()] for l in out.strip().splitlines()], dtype=np.uint64)
    assert got.shape == (len(cases), 4)
    for (s, q, n, t, st), g in zip(cases, got):
        ref = orc.philox([q, n, t, st], [s & 0xFFFFFFFF, s >> 32])
        assert np.array_equal(np.asarray(ref, np.uint64), g), (s, q, n, t, st, ref, g)
