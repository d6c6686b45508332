"""The opt-in two-steps-per-launch path (FDTD_TB=1): the parity cases of the
one-step path rerun through it against the FP64 oracle, and the two paths
against each other on the same inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import workloads
import test_gpu_parity as tp

pytestmark = pytest.mark.gpu


@pytest.fixture
def tb_on(monkeypatch):
    monkeypatch.setenv("FDTD_TB", "1")


@pytest.mark.parametrize("case", [
    "test_cavity_60_full_length",
    "test_multi_tile_ragged_lossy_grid",
    "test_batch_of_uneven_grids",
    "test_cfl_extension_run",
    "test_split_runs_equal_one_run",
    "test_save_load_resume_is_bit_identical",
    "test_full_size_grid_sampled_outputs",
])
def test_parity_case_through_two_step_path(tb_on, case):
    getattr(tp, case)()


def test_two_step_path_agrees_with_one_step_path(monkeypatch):
    w = workloads.random_grid(7, 700, 150, 3, 6, 3, 40, 301, n_probes=12)
    for rd in w["roms"]:
        w["probes"] += [(rd["i0"] - 1, rd["j0"]), (rd["i0"] + rd["a"], rd["j0"] + rd["b"] - 1)]
    res = {}
    for tb in ("0", "1"):
        monkeypatch.setenv("FDTD_TB", tb)
        ctx, _ = tp.gpu_context([w])
        res[tb] = (tp.gpu_run(ctx, [w], 301), ctx.get_fields(0))   # odd count: a trailing single step
    assert tp.rel_l2(res["1"][0], res["0"][0]) < 1e-6
    for a, b in zip(res["1"][1], res["0"][1]):
        assert tp.rel_l2(a, b) < 1e-6
