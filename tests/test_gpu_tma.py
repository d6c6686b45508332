"""The bulk-copy (TMA ring) form of the stencil (FDTD_STENCIL=tma): the
parity cases of the register-prefetch form rerun through it against the FP64
oracle, and both forms against each other bit for bit (they share the
arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import workloads
import test_gpu_parity as tp
import test_gpu_lattice as tl

pytestmark = pytest.mark.gpu


@pytest.fixture
def tma_on(monkeypatch):
    monkeypatch.setenv("FDTD_STENCIL", "tma")


@pytest.mark.parametrize("case", [
    "test_cavity_60_full_length",
    "test_multi_tile_ragged_lossy_grid",
    "test_batch_of_uneven_grids",
    "test_cfl_extension_run",
    "test_random_initial_state_and_tiny_grid",
    "test_split_runs_equal_one_run",
    "test_save_load_resume_is_bit_identical",
    "test_full_size_grid_sampled_outputs",
    "test_batched_layout_parity",
])
def test_parity_case_through_tma_stencil(tma_on, case):
    getattr(tp, case)()


def test_lattice_through_tma_stencil(tma_on):
    tl.test_scaled_lattice_matches_oracle()


@pytest.mark.parametrize("make", [
    lambda: workloads.random_grid(7, 700, 150, 3, 6, 3, 40, 200, n_probes=12),
    lambda: tl.small_lattice(200),
])
def test_tma_and_register_forms_are_bit_identical(monkeypatch, make):
    w = make()
    res = {}
    for form in ("ldg", "tma"):
        monkeypatch.setenv("FDTD_STENCIL", form)
        if "types" in w:
            ctx, _ = tl.lattice_context(w)
        else:
            ctx, _ = tp.gpu_context([w])
        res[form] = (tp.gpu_run(ctx, [w], 200), ctx.get_fields(0))
    np.testing.assert_array_equal(res["tma"][0], res["ldg"][0])
    for a, b in zip(res["tma"][1], res["ldg"][1]):
        np.testing.assert_array_equal(a, b)
