"""The bounds-checked build (liblbm_b300_check.so, compiled with -DLBM_CHECK: the kernels check
their data-dependent indices -- pull sources, cut-link slots, LSQ stencil nodes, upstream and
projection neighbours -- and latch LBM_DEV_BOUNDS instead of leaving an array) runs cases that
cover every closure branch, every population form and a multi-specimen body with no violation, and
gives the same fields, bit for bit, as the normal build."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2606_20646_b300 import lbm, inputs as I
cases = [("random_box_3d", I.random_box(3, 22, 2), 23, "fp64"),
         ("face_touching_3d", I.face_touching_box(3, 32, 3), 23, "fp32"),
         ("shell_bf16", I.shell_3d(32), 23, "bf16s"),
         ("annulus_2d", I.radial_traction_annulus_2d(40), 41, "fp32"),
         ("batch", I.batch_2d(n_spec=4, side=(40, 56), width=192, seed=7, steps=30)[0], 30, "fp32")]
out = {}
for name, p, steps, prec in cases:
    sim = lbm.Simulation(p, precision=prec)
    sim.set_initial().step(steps)
    for k, a in zip("vFu", sim.fields()):
        out[name + "_" + k] = a.cpu().numpy()
    out[name + "_status"] = np.array(sim.sync(raise_on_status=False))
    sim.close()
np.savez(OUT, **out)
"""


def _run(tmp_path, checked):
    from paper_2606_20646_b300 import build
    build.build()
    out = str(tmp_path / ("checked.npz" if checked else "plain.npz"))
    env = dict(os.environ, LBM_B300_CHECK="1" if checked else "0")
    code = f"ROOT = {ROOT!r}\nOUT = {out!r}\n" + SCRIPT
    subprocess.run([sys.executable, "-c", code], env=env, check=True, cwd=ROOT, timeout=600)
    return np.load(out)


def test_checked_build_runs_clean_and_equals_the_normal_build(tmp_path):
    chk = _run(tmp_path, True)
    plain = _run(tmp_path, False)
    for k in chk.files:
        if k.endswith("_status"):
            assert int(chk[k]) == 0, (k, int(chk[k]))
            assert int(plain[k]) == 0, (k, int(plain[k]))
        else:
            assert np.array_equal(chk[k], plain[k]), k
