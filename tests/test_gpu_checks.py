"""The bounds-checked build (librecon_checks.so: every wavefront queue slot and
pixel offset checked before use, failed checks counted and skipped; the
stand-in for a memory checker, which is not available on this GPU pool): on a
spread of cases it gives the oracle's bytes and records no failed check."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, %(root)r)
import numpy as np, torch
import paper_1311_0378_gb300 as rc
rc.LIB_PATH = %(lib)r
import oracle, synth

def dev(a):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda(); torch.cuda.synchronize(); return t

c = rc.recon_init(0, 0, rc.RECON_FLAG_SYNC)
rc.recon_checks(reset=True)
def run(I, J, conn, op=0, params=()):
    for k, v in params:
        rc.check(rc.recon_set_param(c, k, v))
    dI, dJ = dev(I), dev(J)
    rc.check(rc.recon_run_op(c, dI.data_ptr(), dJ.data_ptr(), I.shape[0], I.shape[1], conn, op), "run")
    return dJ.cpu().numpy()
base = synth.workload("single512").tiles[0]
for marker in (synth.HDOME, synth.FILLHOLES):
    I, J = synth.tile_pair(synth.with_marker(base, marker), 1)
    for conn in (4, 8):
        for bh in (32, 128):
            assert (run(I, J, conn, params=((rc.RECON_P_BLOCK_H, bh),)) == oracle.recon(I, J, conn)).all()
        Ic, Jc = 255 - I, 255 - J
        assert (run(Ic, Jc, conn, op=rc.RECON_OP_ERODE) == oracle.recon_erode(Ic, Jc, conn)).all()
    assert (run(I, np.zeros_like(I), 4, op=rc.RECON_OP_FILL_HOLES) == oracle.fill_holes(I, 4)).all()
rng = np.random.default_rng(1)
for H, W in ((37, 53), (300, 1000), (1, 129)):
    I = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    J = np.where(rng.random((H, W)) < 0.02, I, 0).astype(np.uint8)
    for conn in (4, 8):
        assert (run(I, J, conn, params=((rc.RECON_P_SWEEPS, 0), (rc.RECON_P_TMA, 0))) == oracle.recon(I, J, conn)).all()
w = synth.workload("uneven1000")
specs = [s for s in w.tiles[:40] if s.H * s.W <= 1 << 20][:12]
pairs = [synth.tile_pair(s, w.seed) for s in specs]
keep = [(dev(I), dev(J)) for I, J in pairs]
rc.check(rc.recon_batch(c, [(a.data_ptr(), b.data_ptr(), s.H, s.W, s.W, s.conn) for (a, b), s in zip(keep, specs)]))
for (a, b), (I, J), s in zip(keep, pairs, specs):
    assert (b.cpu().numpy() == oracle.recon(I, J, s.conn)).all()
rc.recon_free(c)
en, viol, first = rc.recon_checks()
print("checks", en, viol, first)
'''


def test_checked_build_is_bit_exact_without_violations():
    import paper_1311_0378_gb300.build as b
    lib = b.build(checks=True)
    code = CHILD % {"root": ROOT, "lib": lib}
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [l for l in out.stdout.splitlines() if l.startswith("checks")][-1]
    assert line.split()[1:] == ["1", "0", "0"], line
