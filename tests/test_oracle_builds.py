"""The host-tuned build of the oracle (-O3 -march=native, timed as the CPU
baseline) rounds exactly like the portable build the tests use: ISO C11
forbids contracting a*b + c into a fused multiply-add, so both builds
evaluate the same operations in the same order.  CPU only."""
import subprocess
import sys

SCRIPT = r"""
import sys
import numpy as np
from oracle import oracle as O
from paper_2012_08758_b300 import inputs
if sys.argv[1] == "native":
    O.use_native()
p = O.Params(nx=20, ny=16, nz=12, f0=0.05, sigma=0.6, nu=0.01, eta=0.02, upwind=1)
q = inputs.random_modes_state(20, 16, 12, seed=3, amp=0.2) + inputs.noise_state(20, 16, 12, seed=4, amp=1e-3)
O.run(p, q, 3)
d = O.diagnostics(p, q)
np.save(sys.argv[2], np.concatenate([q.ravel(), np.array(list(d.values()))]))
"""


def test_native_build_gives_the_same_bits(tmp_path):
    import numpy as np
    out = {}
    for kind in ("portable", "native"):
        path = str(tmp_path / f"{kind}.npy")
        subprocess.check_call([sys.executable, "-c", SCRIPT, kind, path], cwd=str(tmp_path.parent),
                              env=_env())
        out[kind] = np.load(path)
    assert np.array_equal(out["portable"], out["native"])


def _env():
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    return dict(os.environ, PYTHONPATH=os.pathsep.join([root, os.environ.get("PYTHONPATH", "")]))
