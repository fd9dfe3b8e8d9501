"""The bounds-checked build (-DVR_DEBUG_BOUNDS) tests every gather and scatter index of the
kernels against its buffer, counts the ones outside and clamps them.  Every renderer, the
adjoint, the probes and the batch run over tiny, ragged and regular volumes of every voxel
type, under views that reach the volume's faces and corners; no index may leave its buffer."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_no_index_leaves_its_buffer():
    from paper_1609_01317_gb300 import build, vr

    build.build()
    lib = build.build(bounds_checked=True)
    env = dict(os.environ, VR_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_bounds_battery.py")],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    counts = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(counts) == 20
    bad = {k: v for k, v in counts.items() if v != 0}
    assert not bad, bad


def test_regular_build_has_no_bounds_counter():
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    r = Renderer(0)
    try:
        with pytest.raises(vr.VrError) as e:
            vr.vr_read_bounds_violations(r.ctx)
        assert e.value.status == 4
    finally:
        r.close()
