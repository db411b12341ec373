"""The FP32-flux stage on grids of awkward shape, on the GPU: against the
FP64 oracle after a run (the mode's 1e-5 bar) with tile rows that start on
Gamma, thin bands, ragged x and a grid narrower than a tile, and the
single-instance kernel against the batch runner's on the same instance (the
same float arithmetic, contracted differently: equal to float rounding)."""
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


def M():
    from paper_2202_11890_gb300 import mprk
    return mprk


@pytest.mark.parametrize("dims,m,wall", [((80, 20, 12, 36), 3, 0), ((80, 17, 16, 36), 2, 1), ((124, 9, 4, 13), 4, 0),
                                         ((8, 3, 4, 5), 2, 0), ((61, 10, 4, 12), 2, 0)])
def test_fp32_flux_steps_close_to_oracle(dims, m, wall):
    """Tile rows that start on Gamma (n1 = 32 at row 32; n1 = 33 at row
    17 + 16), thin bands, ragged x (124 and 61 columns) and a grid narrower
    than a tile (8 columns): 10 slow steps within 1e-5 of the FP64 oracle."""
    mp = M()
    g = W.Grid(*dims)
    q0 = W.gaussian_bumps(g, 41 + m, sigma_cells=3.0)
    cfg, P, dt = pair(g, m, q0=q0, precision=mp.MPRK_FP32FLUX, wall=wall)
    q_or, _ = O.mprk_step(P, q0, 10)
    with mp.Instance(cfg, q0) as inst:
        inst.step(10)
        q_gpu = inst.state()
    err = rel_err(q_gpu, q_or)
    print("fp32flux error per component:", err)
    assert np.all(err < 1e-5), err


@pytest.mark.parametrize("form", ["per_stage", "persistent"])
@pytest.mark.parametrize("scheme", [0, 1])
def test_single_and_batch_kernels_agree(scheme, form, tmp_path):
    """One instance steps with the single-instance stage kernel, its twin
    with a batched step in either form (the per-stage launches, the FP32-flux
    default, or the persistent kernel, chosen here through a tuning entry for
    the instance's size bucket): the states agree to float rounding."""
    mp = M()
    g = W.Grid(124, 20, 12, 36)
    q0 = W.gaussian_bumps(g, 7, sigma_cells=3.0)
    cfg, P, dt = pair(g, 3, q0=q0, precision=mp.MPRK_FP32FLUX, scheme=scheme)
    mp.mprk_tune_clear()
    if form == "persistent":
        bucket = int(np.floor(np.log2(g.nx * g.nz)))
        path = tmp_path / "t.json"
        path.write_text('{"gpu": "%s", "entries": [{"precision": 1, "bucket": %d, "group": 2, '
                        '"ctas_per_sm": 0, "ms": 1}]}' % (torch.cuda.get_device_name(0), bucket))
        mp.mprk_tune_load(str(path))
        assert mp.mprk_tune_lookup(1, g.nx * g.nz)["tiles_per_item"] == 2
    try:
        with mp.Instance(cfg, q0) as a, mp.Instance(cfg, q0) as b:
            for _ in range(3):
                a.step(1)
                mp.mprk_step_batch([b.h], 1)
                err = rel_err(a.state(), b.state())
                print(form, "single vs batch:", err)
                assert np.all(err < 1e-6), err
    finally:
        mp.mprk_tune_clear()
