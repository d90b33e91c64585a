"""The tensor-core FIFO sweep (VI_KERNEL_TENSOR) against the oracle: full solves
at the oracle's stopping iteration on shapes that span several tiles and a
ragged last tile, every supported pipeline length and demand range, and the
4.08M-state FIFO instance on sampled states in the benchmark's launch
configuration."""
import numpy as np
import pytest
import torch

import workloads
from workloads import FIFO, LIFO

pytestmark = pytest.mark.gpu

vi = pytest.importorskip("paper_2303_10672_b300")
from gpu_helpers import Handle, compare_values, V_RTOL  # noqa: E402
from test_gpu_parity import SMALL, sampled_backup_parity, solve_parity  # noqa: E402

C1 = (3.0, 1.0, 5.0, 7.0, 0.0)
C2 = (2.0, 1.5, 6.0, 4.0, 1.0)


def tc_cases():
    sp = workloads.single_product
    out = [
        sp(3, 2, 5, C1, workloads.poisson_pmf(2.0, 10), 0.9, FIFO),          # 216 states, 2 tiles, ragged
        sp(4, 2, 7, C2, workloads.negbin_pmf(4.0, 9.0, 20), 0.95, FIFO),     # 4096 states, 32 tiles
        sp(3, 3, 9, C1, workloads.poisson_pmf(4.0, 20), 0.9, FIFO),          # 10^4 states, 84 tiles, ragged
        sp(2, 2, 31, C2, workloads.poisson_pmf(8.0, 30), 0.9, FIFO),         # Q+1 = 32 columns
        sp(3, 2, 4, C1, workloads.poisson_pmf(1.0, 3), 0.9, FIFO),           # Dmax < 16
        sp(2, 2, 6, C1, workloads.poisson_pmf(20.0, 100), 0.9, FIFO),        # Dmax = 100
        sp(2, 4, 3, C2, workloads.poisson_pmf(1.5, 9), 0.95, FIFO),          # long pipeline
        sp(3, 2, 1, C1, workloads.poisson_pmf(0.7, 4), 0.9, FIFO),           # Q+1 = 2
    ]
    out += [x for x in SMALL if x.issuing == FIFO and x.products[0].L >= 2 and x.products[0].Q + 1 <= 32
            and x.products[0].m >= 2 and x.products[0].dmax >= 1 and x.products[0].Q >= 1]
    return out


TC = tc_cases()


def _ids(insts):
    return [f"{i}-m{x.products[0].m}L{x.products[0].L}Q{x.products[0].Q}D{x.products[0].dmax}"
            for i, x in enumerate(insts)]


@pytest.mark.parametrize("inst", TC, ids=_ids(TC))
def test_tensor_solve_parity(inst):
    solve_parity(inst, "fp32", kernel=vi.VI_KERNEL_TENSOR)


def test_tensor_config2_full_size_sampled():
    sampled_backup_parity(workloads.config2(), 3, 300, 2, "fp32", kernel=vi.VI_KERNEL_TENSOR)


def test_tensor_matches_cuda_core_kernel_on_config2():
    """Both factorised kernels after the same number of sweeps: values agree to
    FP32 accuracy and the policies differ only on near-ties."""
    inst = workloads.config2()
    with Handle(inst, precision="fp32", kernel=vi.VI_KERNEL_TENSOR) as T, \
            Handle(inst, precision="fp32", kernel=vi.VI_KERNEL_GROUP) as C:
        Vt, pt, it = T.solve(0.0, 6)
        Vc, pc, ic = C.solve(0.0, 6)
        err = compare_values(T.v_abs(Vt, it), C.v_abs(Vc, ic))
        assert err <= 1e-6, err
        diff = (pt != pc).sum().item()
        assert diff <= 1e-4 * pt.numel(), diff


def test_tensor_option_rejected_where_unsupported():
    lifo = workloads.single_product(3, 2, 5, C1, workloads.poisson_pmf(2.0, 10), 0.9, LIFO)
    l1 = workloads.single_product(3, 1, 5, C1, workloads.poisson_pmf(2.0, 10), 0.9, FIFO)
    big_q = workloads.single_product(2, 2, 40, C1, workloads.poisson_pmf(2.0, 10), 0.9, FIFO)
    for inst, prec in ((lifo, "fp32"), (l1, "fp32"), (big_q, "fp32"), (TC[0], "fp64"), (TC[0], "fp32_single")):
        with pytest.raises(vi.ViError):
            with Handle(inst, precision=prec, kernel=vi.VI_KERNEL_TENSOR):
                pass


def test_tensor_extraction_and_backup_modes():
    """vi_backup (plain mode) with the tensor kernel equals the solve's next sweep,
    and the extraction writes the same policy as the plain backup."""
    inst = TC[2]
    with Handle(inst, precision="fp32", kernel=vi.VI_KERNEL_TENSOR) as H:
        V, pol, info = H.solve(0.0, 5)
        V6, pol6, info6 = H.solve(0.0, 6)
        out = torch.empty_like(V)
        pb = torch.empty_like(pol)
        vi.vi_backup(H.h, V, out, pb)
        torch.cuda.synchronize()
        assert torch.equal(out, V6)
        assert torch.equal(pb, pol)   # extraction of the 5-sweep solve = argmax from V_5


def test_bounded_wait_reports_and_context_survives():
    """The tensor-core kernel's wait for its MMAs is bounded: with the test hook
    that withholds the MMAs, the sweep reports VI_ECUDA instead of hanging, and
    the handle works normally afterwards."""
    inst = TC[2]
    with Handle(inst, precision="fp32", kernel=vi.VI_KERNEL_TENSOR) as H:
        V, pol, info = H.solve(0.0, 2)
        out = torch.empty_like(V)
        vi.vi_problem_set_option(H.h, vi.VI_OPT_TEST_STALL, 1)
        with pytest.raises(vi.ViError) as e:
            vi.vi_backup(H.h, V, out, None)
        assert e.value.status == vi.VI_ECUDA
        with pytest.raises(vi.ViError) as e:
            H.solve(1e-4, 20)
        assert e.value.status == vi.VI_ECUDA
        vi.vi_problem_set_option(H.h, vi.VI_OPT_TEST_STALL, 0)
        V3, pol3, info3 = H.solve(0.0, 3)
        vi.vi_backup(H.h, V3, out, None)
        torch.cuda.synchronize()
    with Handle(inst, precision="fp32", kernel=vi.VI_KERNEL_TENSOR) as F:
        V4, pol4, info4 = F.solve(0.0, 3)
    assert torch.equal(V3, V4) and torch.equal(pol3, pol4)
