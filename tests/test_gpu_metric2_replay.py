"""The GPU's Algorithm-1 runs on the 32^3 workload (nearest, no CTF, SNR
0.1, batch 100, 5 epochs) follow the oracle's relative-error curves.

tests/golden/metric2_m32_curves.txt holds, for the plain, Algorithm-1 and
precomputed-D arms, the relative error |v - v*| / |v*| after every iteration
of the literal FP64 oracle, written by tests/golden/make_metric2_curves.py
(oracle only).  The GPU replays the same inputs, start, permutations and
probe seeds through the library: the accepted step sizes must be the same at
every iteration, the first epoch's errors within 1e-4 (relative) of the
oracle's and all 50 within 1e-3.  The ordering of the arms on this workload
(plain SGD ending lowest, the precomputed D highest) is then the method's,
not the kernels'.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_curves():
    rows = {}
    for line in open(os.path.join(GOLDEN, "metric2_m32_curves.txt")):
        if line.startswith("#") or not line.strip():
            continue
        setting, arm, k, e, eta = line.split()
        rows.setdefault((setting, arm), []).append((int(k), float(e), float(eta)))
    return rows


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, GOLDEN)
    import make_metric2_curves as mk
    from paper_2311_16100_gb300.ops import Handle
    S = mk.problem()
    h = Handle(0)
    yield mk, S, h
    h.close()


@pytest.mark.parametrize("arm,mode", [("plain", "plain"), ("hutchinson", "hutchinson"),
                                      ("precomputed", "fixed")])
def test_gpu_curve_follows_oracle(setup, arm, mode):
    from paper_2311_16100_gb300.ops import Geometry, SGDState
    mk, S, h = setup
    P = mk.P
    want = read_curves()[("batch100", arm)]
    M, r, N, B = S["M"], S["r"], len(S["R"]), P["B"]
    d = torch.device("cuda")
    geom = Geometry(M, r, "nearest", None)
    x = torch.from_numpy(S["x"]).to(d)
    R = torch.from_numpy(S["R"]).to(d)
    vstar = torch.from_numpy(S["vstar"].astype(np.complex64)).to(d)
    D = None
    if mode == "fixed":
        D = h.precompute_preconditioner(geom, R, None, B=B, n_epochs=1, lam=S["lam"],
                                        n_probes=P["K"], seed=P["seed"] + 13)
    st = SGDState(torch.from_numpy(S["v0"]).to(d), mode=mode, alpha=S["alpha"],
                  eta0=P["eta0"], beta=P["beta"], armijo_c=P["c"], n_probes=P["K"],
                  seed=P["seed"] + 11, D=D)
    got = []
    for ep in range(P["epochs"]):
        perm = torch.from_numpy(S["perms"][ep]).to(d)
        xp, Rp = x[perm].contiguous(), R[perm].contiguous()
        for s in range(0, N, B):
            h.precond_sgd_step(geom, st, xp[s:s + B], Rp[s:s + B], None, S["lam"], N / B)
            got.append((float(h.rel_err(geom, st.v, vstar)), float(st.scalars[0])))
    assert len(got) == len(want) == 50
    for i, ((e, eta), (k, ew, etaw)) in enumerate(zip(got, want)):
        assert eta == etaw, (arm, k, eta, etaw)
        tol = 1e-4 if k <= N // B else 1e-3
        assert abs(e - ew) <= tol * ew, (arm, k, e, ew)
