"""Library calls on several streams at once, through the C-ABI.  The device memory
pool hands blocks back in stream order: a block freed while kernels still use it
(the contraction's packed operands, the leaves of destroyed halves) carries an
event of its stream, and a request from another stream waits for that event.
Circuits of equal sizes on two streams therefore trade the same blocks while their
kernels run; every result must still be the oracle's."""
import threading

import numpy as np
import pytest

import oracle
from oracle import circuit as oc
import paper_1802_06952_gb300 as sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
SHAPE = (4, 5, 16, 2)  # rows, cols, depth, cut row: 10 + 10 qubits


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06952_gb300 import build
    build.build()
    sim.lib()
    torch.cuda.set_device(0)
    yield
    sim.sim_release_cache()


@pytest.fixture(scope="module")
def refs():
    R, C, d, b = SHAPE
    out = {}
    for seed in range(8):
        gates, plan = oc.grid_cut(R, C, d, seed, b)
        out[seed] = oracle.statevector(R * C, gates).reshape(1 << plan.n_l, 1 << plan.n_u)
    return out


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def run_one(seed, stream, out):
    """Build, cut, evolve, contract on `stream` into `out`; destroy without waiting."""
    R, C, d, b = SHAPE
    circ = sim.sim_build_circuit(R, C, d, seed, b)
    plan, c, copies, nu, nl = sim.sim_cut(circ, b)
    h = sim.sim_evolve_halves(plan, sim.SIM_C64, 0, copies, stream=stream)
    sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, False, out, stream=stream)
    sim.sim_destroy_halves(h)
    sim.sim_destroy_cut(plan)
    sim.sim_destroy_circuit(circ)


def test_contraction_in_flight_while_another_stream_reuses_the_pool(refs):
    """Stream A's contraction is enqueued and its buffers freed; stream B, with A's
    work still queued behind a long sweep, immediately asks for blocks of the same
    sizes.  Both outputs are the oracle's."""
    R, C, d, b = SHAPE
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    oa = torch.zeros((1 << ((R - b) * C), 1 << (b * C)), dtype=torch.complex64, device="cuda")
    ob = torch.zeros_like(oa)
    for _ in range(3):
        run_one(0, sa, oa)
        run_one(1, sb, ob)
        torch.cuda.synchronize()
        assert rel(oa.cpu().numpy(), refs[0]) <= TOL
        assert rel(ob.cpu().numpy(), refs[1]) <= TOL


def test_two_threads_two_streams(refs):
    """Two host threads, each on its own stream, run circuits of equal sizes
    back to back without waiting between them; each checks its outputs."""
    R, C, d, b = SHAPE
    errors = []

    def worker(tid):
        try:
            st = torch.cuda.Stream()
            outs = [torch.zeros((1 << ((R - b) * C), 1 << (b * C)), dtype=torch.complex64, device="cuda")
                    for _ in range(4)]
            seeds = [(tid * 4 + i) % 8 for i in range(4)]
            for rep in range(3):
                for o, s in zip(outs, seeds):
                    run_one(s, st, o)
                st.synchronize()
                for o, s in zip(outs, seeds):
                    e = rel(o.cpu().numpy(), refs[s])
                    if e > TOL:
                        errors.append((tid, rep, s, e))
        except Exception as ex:  # reported below
            errors.append((tid, repr(ex)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in threads)
    assert not errors, errors
