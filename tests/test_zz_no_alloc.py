"""nb_force_static: the force call for callers that cannot allocate device memory
(for example code inside another framework's memory pool or a loop that must not
allocate once running).  Checked through the C ABI against the oracle's direct
sum on the same state, with the parity gate of the other GPU tests, on two calls
in a row (the fixed scratch keeps the first call's contents), and against
nb_force on the same instant.  This file is named to be collected last."""
import ctypes as C

import numpy as np
import pytest

import oracle as orc
from gpu_common import assert_force_close
from oracle import parity

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_static_force_matches_oracle_and_nb_force_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_1312_1789_b300 import build, ics, nb
    build.build()
    L = nb.lib()
    n = 3000
    m, x, v = ics.plummer(n - 2, 31)
    mb, xb, vb = ics.bh_circular_pair(0.005, 0.1)
    m, x, v = np.concatenate([m, mb]), np.concatenate([x, xb]), np.concatenate([v, vb])
    eps2 = np.concatenate([np.full(n - 2, 1e-8), np.zeros(2)])
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.choice(n - 2, 1200, replace=False), [n - 2, n - 1]])).astype(np.int32)
    stream = torch.cuda.current_stream()
    for prec in (nb.NB_FP64, nb.NB_MIXED):
        for order in (6, 8):
            ctx = nb.NBody(n, order, 0.0, prec)
            ctx.set_stream(stream)
            ctx.set_softening(np.sqrt(eps2))
            ctx.set_particles(m, x, v)
            S = ctx.get_state()
            ctx.predict(0.0)
            ctx.force(idx)
            via_ctx = ctx.get_force(len(idx))
            ctx.close()
            # the oracle on the very state handed to the static call (no prediction)
            ref = orc.force(m, eps2, S["x"], S["v"], S["d"][:, 0], S["d"][:, 1] if order == 8 else None,
                            order=order, idx=idx, nthreads=16)
            dev = {k: torch.from_numpy(np.ascontiguousarray(a)).cuda()
                   for k, a in (("m", m), ("eps2", eps2), ("x", S["x"]), ("v", S["v"]),
                                ("a", S["d"][:, 0]), ("j", S["d"][:, 1]))}
            didx = torch.from_numpy(idx).cuda()
            nc = 3 * (order // 2) + 2
            out = torch.empty((nc, len(idx)), dtype=torch.float64, device="cuda")
            for call in range(2):
                out.fill_(float("nan"))
                rc = L.nb_force_static(order, prec, n, _ptr(dev["m"]), _ptr(dev["eps2"]), _ptr(dev["x"]),
                                       _ptr(dev["v"]), _ptr(dev["a"]), _ptr(dev["j"]), _ptr(didx), len(idx),
                                       _ptr(out), C.c_void_p(stream.cuda_stream))
                assert rc == nb.NB_OK, L.nb_last_error(None)
                got = out.cpu().numpy()
                G = {"acc": got[0:3].T, "jerk": got[3:6].T, "pot": got[3 * (order // 2)]}
                if order >= 6:
                    G["snap"] = got[6:9].T
                if order >= 8:
                    G["crackle"] = got[9:12].T
                assert_force_close(G, ref, order, prec, f"static call {call}, precision {prec}, order {order}")
                # nb_force on the same instant: both lie within the gate of the
                # oracle, so they differ by at most twice its bound
                st = parity.force_parity(G, dict(via_ctx, absum=ref["absum"]), order, prec)
                assert all(r["worst"] <= 2.0 for r in st.values()), (call, prec, order, st)


def test_static_force_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_1312_1789_b300 import build, nb
    build.build()
    L = nb.lib()
    n = nb.NB_STATIC_MAX_N + 1
    buf = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    idx = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    rc = L.nb_force_static(6, nb.NB_MIXED, n, p, p, p, p, p, None, C.c_void_p(idx.data_ptr()), 1,
                           C.c_void_p(out.data_ptr()), None)
    assert rc == nb.NB_ERR_ARG
    assert str(nb.NB_STATIC_MAX_N).encode() in L.nb_last_error(None)
