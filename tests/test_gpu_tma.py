"""CGS2 sweeps with the basis staged by the bulk-copy (TMA) engine (opt-in,
PP_TMA_CGS) against the plain sweeps, through the C-ABI.

Both compute the same projections on the same rows in different orders, so
they agree to rounding.  Each run happens in a child process because the
switch is read once.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, %r)
from paper_1806_08020_gb300 import inputs, pp
out = {}
for prec, dt in ((1, torch.float32),):
    for n, j in ((4099, 33), (100003, 51), (20000, 128), (64, 3)):
        rng = np.random.default_rng(n + j + prec)
        Q, _ = np.linalg.qr(rng.standard_normal((n, j)))
        w = rng.standard_normal(n) + Q @ rng.standard_normal(j) * 10
        ctx = pp.pp_create(inputs.diagonal(np.ones(n)), stream=torch.cuda.current_stream().cuda_stream,
                           precision=prec)
        ldv = (n + 31) // 32 * 32
        Vd = torch.zeros((j, ldv), dtype=dt, device="cuda")
        Vd[:, :n] = torch.tensor(Q.T, dtype=dt)
        wd = torch.tensor(w, dtype=dt, device="cuda")
        vd = torch.empty(n, dtype=dt, device="cuda")
        h = pp.pp_orthogonalize(ctx, Vd.data_ptr(), ldv, j, wd.data_ptr(), vd.data_ptr())
        out[f"{prec}_{n}_{j}"] = [h.tolist(), vd.double().cpu().numpy().tolist()]
json.dump(out, sys.stdout)
""" % ROOT


def _run(no_tma: bool):
    env = dict(os.environ)
    env.pop("PP_TMA_CGS", None)
    if not no_tma:
        env["PP_TMA_CGS"] = "1"
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout)


@pytest.mark.gpu
def test_tma_sweeps_match_plain_sweeps():
    tma = _run(False)
    plain = _run(True)
    for key in tma:
        prec = int(key.split("_")[0])
        tol = 1e-12 if prec == 0 else 1e-5
        h_t, v_t = (np.array(x) for x in tma[key])
        h_p, v_p = (np.array(x) for x in plain[key])
        assert np.abs(h_t - h_p).max() <= tol * np.abs(h_p).max(), key
        assert np.abs(v_t - v_p).max() <= tol * max(1.0, np.abs(v_p).max()) * 10, key


@pytest.mark.gpu
def test_staged_sweep_wait_expiry_is_reported_and_recoverable():
    """Failure path of the staged sweeps without a GPU fault: with the copies
    withheld (a barrier that nothing arms) every bounded wait runs out, the
    call returns PP_ETIMEOUT, and the same context then computes correctly."""
    import time

    import torch

    import oracle as O
    from paper_1806_08020_gb300 import inputs, pp
    n, j = 100003, 21
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((n, j)))
    Q = Q.astype(np.float32).astype(np.float64)
    w = (rng.standard_normal(n) + Q @ rng.standard_normal(j)).astype(np.float32).astype(np.float64)
    ctx = pp.pp_create(inputs.diagonal(np.ones(n)), stream=torch.cuda.current_stream().cuda_stream,
                       precision=pp.PP_FP32)
    ldv = (n + 31) // 32 * 32
    Vd = torch.zeros((j, ldv), dtype=torch.float32, device="cuda")
    Vd[:, :n] = torch.tensor(Q.T, dtype=torch.float32)
    vd = torch.empty(n, dtype=torch.float32, device="cuda")
    pp.pp_debug_stall_sweeps(ctx, 1)
    wd = torch.tensor(w, dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    with pytest.raises(pp.PPError) as e:
        pp.pp_orthogonalize(ctx, Vd.data_ptr(), ldv, j, wd.data_ptr(), vd.data_ptr())
    assert e.value.status == pp.PP_ETIMEOUT
    assert time.perf_counter() - t0 < 60
    wd = torch.tensor(w, dtype=torch.float32, device="cuda")
    h = pp.pp_orthogonalize(ctx, Vd.data_ptr(), ldv, j, wd.data_ptr(), vd.data_ptr())
    _, href = O.cgs2(Q, w, O.Counters())
    assert np.abs(h[:j] - href).max() <= 16 * 2.0**-24 * np.linalg.norm(w)
