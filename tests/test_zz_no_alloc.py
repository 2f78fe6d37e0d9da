"""qbf_solve_noalloc against qbf_solve, through the C ABI.

qbf_solve_noalloc serves callers that cannot allocate GPU memory (a process
that reserved the whole device for its own pool, a plug-in inside an
application that owns the memory budget, a service that cannot take the
synchronisation an allocation may cause).  It must give exactly the answer of
qbf_solve -- the tests' tolerance for both integer and certified float Q is
equality -- and keep giving it when called again on its shared scratch.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2310_19373_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2310_19373_gb300 import _binding as qb  # noqa: E402


def _fields(r):
    k = r.top_k
    return (r.top_k, list(r.topk_value[:k]), list(r.topk_index[:k]), r.min_value, r.argmin,
            r.scale_bits, r.error_bound)


@pytest.mark.parametrize("case", ["n20_f64_top8", "n32_int_top2", "n16_f32", "n36_int16"])
def test_noalloc_matches_solve_twice(case):
    if case == "n20_f64_top8":
        Q, k = inputs.config_n20_f64(0), 8
    elif case == "n32_int_top2":
        Q, k = inputs.config_n32_int(0), 2
    elif case == "n16_f32":
        Q, k = inputs.gaussian_f32(16, seed=4), 3
    else:
        Q, k = inputs.uniform_int(36, seed=2, lo=-50, hi=50, dtype=np.int16), 1
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    code = qb.dtype_code(Qd)
    n = Q.shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    opt = qb.make_options(top_k=k)
    ref = _fields(qb.qbf_solve(Qd.data_ptr(), n, code, opt, stream))
    for _ in range(2):
        got = _fields(qb.qbf_solve_noalloc(Qd.data_ptr(), n, code, opt, stream))
        assert got == ref


def test_noalloc_rejects_oversized_problem():
    Qd = torch.from_numpy(inputs.config_n40_f32(0)).cuda()
    with pytest.raises(qb.QbfError) as e:
        qb.qbf_solve_noalloc(Qd.data_ptr(), 40, qb.QBF_F32, qb.make_options(),
                             torch.cuda.current_stream().cuda_stream)
    assert e.value.status == qb.QBF_EINVAL
    assert "36" in str(e.value)


def test_noalloc_float_walk_form_fields():
    """Float Q at 24 <= n <= 36, where qbf_solve's automatic form is the
    deferred FP32-image walk: the answer equals AUTO's, and the image fields
    (sigma, window, candidates) equal those of qbf_solve's int32 walk, which is
    the walk this call runs."""
    Q = inputs.gaussian_f32(30, seed=6)
    Qd = torch.from_numpy(Q).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    auto = qb.qbf_solve(Qd.data_ptr(), 30, qb.QBF_F32, qb.make_options(top_k=2), stream)
    split = qb.qbf_solve(Qd.data_ptr(), 30, qb.QBF_F32,
                         qb.make_options(top_k=2, variant=qb.QBF_VARIANT_SPLIT), stream)
    for _ in range(2):
        got = qb.qbf_solve_noalloc(Qd.data_ptr(), 30, qb.QBF_F32, qb.make_options(top_k=2), stream)
        assert _fields(got)[:5] == _fields(auto)[:5]
        assert _fields(got) == _fields(split)


def test_noalloc_window_limit():
    """An exact top-2 of the zero matrix ties every state: more than the 2^16
    candidate states this call holds (qbf_solve, with room for 2^22, answers)."""
    Qd = torch.zeros((20, 20), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(qb.QbfError) as e:
        qb.qbf_solve_noalloc(Qd.data_ptr(), 20, qb.QBF_I32, qb.make_options(top_k=2), stream)
    assert e.value.status == qb.QBF_EOVERFLOW and "2^16" in str(e.value)
    r = qb.qbf_solve(Qd.data_ptr(), 20, qb.QBF_I32, qb.make_options(top_k=2), stream)
    assert list(r.topk_index[:2]) == [0, 1]


def test_noalloc_sets_nothing_aside_after_its_first_call():
    """After a first call on the device, further calls leave the device's free
    memory unchanged."""
    Q = inputs.uniform_int(22, seed=3, lo=-40, hi=40)
    Qd = torch.from_numpy(Q).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    first = _fields(qb.qbf_solve_noalloc(Qd.data_ptr(), 22, qb.QBF_I32, qb.make_options(),
                                         stream))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _fields(qb.qbf_solve_noalloc(Qd.data_ptr(), 22, qb.QBF_I32, qb.make_options(),
                                            stream)) == first
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
