"""The persistent batched step (mprk_step_batch): each instance of an uneven
batch ends bitwise equal to the same instance stepped alone with mprk_step,
and the bounded stage waits give up with a timeout status instead of
hanging when a stage never completes."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2202_11890_gb300 import workloads as W
from pairs import oracle_threads, pair, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_11890_gb300 import build
    build.build()
    oracle_threads()


def uneven(count, seed, precision=0):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        nx = int(rng.integers(8, 140))
        nB = int(rng.integers(4, 17))
        nS = int(rng.integers(2, 40))
        nF = int(rng.integers(2, 40))
        m = int(rng.choice([1, 2, 3, 4, 8]))
        g = W.Grid(nx, nS, nB, nF)
        q = W.gaussian_bumps(g, seed * 100 + j, sigma_cells=2.5)
        cfg, P, dt = pair(g, m, q0=q, precision=precision)
        out.append((cfg, P, q))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_each_instance_alone(precision):
    """FP64: bitwise (both kernels run the same non-inlined tile body).
    FP32 flux: within the mode's tolerance (the tile is inlined into each
    kernel, which may contract float operations differently)."""
    from paper_2202_11890_gb300 import mprk as M
    cases = uneven(14, 3 + precision, precision)
    steps = 3
    alone = []
    for cfg, P, q in cases:
        with M.Instance(cfg, q) as inst:
            inst.step(steps)
            alone.append(inst.state())
    insts = [M.Instance(cfg, q) for cfg, P, q in cases]
    try:
        M.mprk_step_batch([i.h for i in insts], steps)
        for i, ref in zip(insts, alone):
            out = i.state()
            if precision == 0:
                assert np.array_equal(out, ref)
            else:
                assert np.all(rel_err(out, ref) < 1e-5), rel_err(out, ref)
            assert i.status() == 0
            assert i.diagnostics()[14] == steps
    finally:
        for i in insts:
            i.close()


def test_batch_matches_oracle():
    from paper_2202_11890_gb300 import mprk as M
    cases = uneven(5, 9)
    insts = [M.Instance(cfg, q) for cfg, P, q in cases]
    try:
        M.mprk_step_batch([i.h for i in insts], 1)
        for (cfg, P, q), i in zip(cases, insts):
            q_or, _ = O.mprk_step(P, q)
            assert np.all(rel_err(i.state(), q_or) < 1e-12)
    finally:
        for i in insts:
            i.close()


def test_batch_wait_times_out_without_hanging():
    """A stage whose tiles never report completion: the waiting tiles give up
    after the cycle limit, the status word reads MPRK_ETIMEOUT, and the
    device stays usable."""
    from paper_2202_11890_gb300 import mprk as M
    cases = uneven(3, 21)
    insts = [M.Instance(cfg, q) for cfg, P, q in cases]
    try:
        rc = M.mprk_batch_test_withhold([i.h for i in insts], 0, 1, 200_000_000)
        assert rc == 0
        torch.cuda.synchronize()
        assert insts[0].status() == M.MPRK_ETIMEOUT
    finally:
        for i in insts:
            i.close()
    # the context still works: a fresh instance steps and matches the oracle
    cfg, P, q = uneven(1, 22)[0]
    with M.Instance(cfg, q) as inst:
        inst.step(1)
        q_or, _ = O.mprk_step(P, q)
        assert np.all(rel_err(inst.state(), q_or) < 1e-12)


def test_batch_rejects_mixed_precisions():
    from paper_2202_11890_gb300 import mprk as M
    a = uneven(1, 30, 0)[0]
    b = uneven(1, 31, 1)[0]
    ia, ib = M.Instance(a[0], a[2]), M.Instance(b[0], b[2])
    try:
        with pytest.raises(M.MprkError) as ei:
            M.mprk_step_batch([ia.h, ib.h], 1)
        assert ei.value.code == M.MPRK_EINVAL
    finally:
        ia.close()
        ib.close()


def test_batch_rejects_an_instance_listed_twice():
    """Two work items on one instance's buffers in one launch would race:
    the batch and the tuner refuse the list, and the instance still steps."""
    from paper_2202_11890_gb300 import mprk as M
    cfg, P, q = uneven(1, 33, 0)[0]
    with M.Instance(cfg, q) as inst:
        for call in (lambda: M.mprk_step_batch([inst.h, inst.h], 1),
                     lambda: M.mprk_batch_tune([inst.h, inst.h], reps=1)):
            with pytest.raises(M.MprkError) as ei:
                call()
            assert ei.value.code == M.MPRK_EINVAL
        M.mprk_step_batch([inst.h], 1)
        q_or, _ = O.mprk_step(P, q)
        assert np.all(rel_err(inst.state(), q_or) < 1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_launch_leaves_states_and_results_unchanged(precision, tmp_path):
    """mprk_batch_tune restores every state and step count it advanced, its
    choice lands in the table (and in a saved file keyed by this GPU's
    name), and batched steps with the tuned launch equal those with the
    default launch bitwise: the choice moves work, not arithmetic."""
    from paper_2202_11890_gb300 import mprk as M
    M.mprk_tune_clear()
    cases = uneven(6, 11 + precision, precision)
    a = [M.Instance(cfg, q) for cfg, P, q in cases]
    b = [M.Instance(cfg, q) for cfg, P, q in cases]
    try:
        M.mprk_step_batch([i.h for i in b], 2)  # default launch
        before = [i.state() for i in a]
        best = M.mprk_batch_tune([i.h for i in a], reps=2)
        if best["tiles_per_item"] == 0:  # the per-stage form (FP32 flux only)
            assert precision == 1 and best["ctas_per_sm"] in (1, 2, 4)  # instance groups
        else:
            assert best["tiles_per_item"] in (1, 2, 4, 8, 16) and 1 <= best["ctas_per_sm"] <= 3
        assert best["ms_per_step"] > 0
        for i, q in zip(a, before):
            assert np.array_equal(i.state(), q) and i.info()["cell_stages_per_step"] > 0
        mean = np.mean([c.nx * (c.nz_S + c.nz_B + c.nz_F) for c, P, q in cases])
        look = M.mprk_tune_lookup(precision, mean)
        assert look["tuned"] and look["tiles_per_item"] == best["tiles_per_item"]
        M.mprk_step_batch([i.h for i in a], 2)  # tuned launch
        for x, y in zip(a, b):
            if precision == 0 or best["tiles_per_item"] == 0:  # same form and tile code as the default
                assert np.array_equal(x.state(), y.state())
            else:  # the persistent kernel's float tile against the per-stage one's
                assert np.all(rel_err(x.state(), y.state()) < 1e-6)
        path = tmp_path / "tune.json"
        M.mprk_tune_save(str(path))
        assert torch.cuda.get_device_name(0) in path.read_text()
        M.mprk_tune_clear()
        M.mprk_tune_load(str(path))
        assert M.mprk_tune_lookup(precision, mean) == look
    finally:
        for i in a + b:
            i.close()
        M.mprk_tune_clear()


@pytest.mark.parametrize("groups", [1, 2, 4])
def test_per_stage_form_groups_match_each_instance_alone(groups, tmp_path):
    """The per-stage form of FP32-flux batches with 1, 2 or 4 instance
    groups (each group's launches on a stream of its own, forked from and
    joined into the batch's stream), forced through a tuning entry: uneven
    instances with m from 1 to 8 (so groups end their stages at different
    launches, and some launches cover one instance) end within float
    rounding of each instance stepped alone, and report no status."""
    from paper_2202_11890_gb300 import mprk as M
    cases = uneven(9, 40 + groups, 1)
    steps = 3
    alone = []
    for cfg, P, q in cases:
        with M.Instance(cfg, q) as inst:
            inst.step(steps)
            alone.append(inst.state())
    mean = np.mean([c.nx * (c.nz_S + c.nz_B + c.nz_F) for c, P, q in cases])
    bucket = int(np.floor(np.log2(mean)))
    path = tmp_path / "t.json"
    path.write_text('{"gpu": "%s", "entries": [{"precision": 1, "bucket": %d, "group": 0, '
                    '"ctas_per_sm": %d, "ms": 1}]}' % (torch.cuda.get_device_name(0), bucket, groups))
    M.mprk_tune_clear()
    M.mprk_tune_load(str(path))
    look = M.mprk_tune_lookup(1, mean)
    assert look["tiles_per_item"] == 0 and look["ctas_per_sm"] == groups
    insts = [M.Instance(cfg, q) for cfg, P, q in cases]
    try:
        M.mprk_step_batch([i.h for i in insts], steps)
        for i, ref in zip(insts, alone):
            err = rel_err(i.state(), ref)
            assert np.all(err < 1e-6), err
            assert i.status() == 0
            assert i.diagnostics()[14] == steps
    finally:
        for i in insts:
            i.close()
        M.mprk_tune_clear()
