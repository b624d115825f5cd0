"""NULL handles and NULL output pointers through the C ABI (no GPU): every entry point that takes a
state or batch answers a NULL one with TUCKER_EINVAL (the counts with -1, the error text with
"null state", destroy with nothing) instead of touching memory, as the header documents."""

import ctypes

import pytest

EINVAL = 1


@pytest.fixture(scope="module")
def lib():
    from paper_2308_16395_gb300 import build as b

    b.build()
    import paper_2308_16395_gb300 as p

    return p.load_library()


def test_state_entry_points_refuse_a_null_state(lib):
    d = ctypes.c_double()
    i64 = (ctypes.c_int64 * 8)()
    calls = {
        "tucker_stream_update": lambda: lib.tucker_stream_update(None, None, None),
        "tucker_stream_update_block": lambda: lib.tucker_stream_update_block(None, None, 2, None),
        "tucker_stream_update_host": lambda: lib.tucker_stream_update_host(None, None, None),
        "tucker_reconstruct": lambda: lib.tucker_reconstruct(None, 0, 1, None, None),
        "tucker_reconstruct_noalloc": lambda: lib.tucker_reconstruct_noalloc(None, 0, 1, None, None),
        "tucker_error_norm": lambda: lib.tucker_error_norm(None, ctypes.byref(d), ctypes.byref(d)),
        "tucker_error_norm_async": lambda: lib.tucker_error_norm_async(None, None, None),
        "tucker_get_ranks": lambda: lib.tucker_get_ranks(None, i64, None),
        "tucker_get_step_info": lambda: lib.tucker_get_step_info(None, None),
        "tucker_get_step_log": lambda: lib.tucker_get_step_log(None, 0, 1, None),
        "tucker_replay_next": lambda: lib.tucker_replay_next(None, None),
        "tucker_orthogonality_error": lambda: lib.tucker_orthogonality_error(None, None),
        "tucker_restore_orthogonality": lambda: lib.tucker_restore_orthogonality(None, None, None),
        "tucker_test_stall_next": lambda: lib.tucker_test_stall_next(None),
        "tucker_recompress": lambda: lib.tucker_recompress(None, 1e-3, None, None),
        "tucker_copy_factor": lambda: lib.tucker_copy_factor(None, 0, None),
        "tucker_copy_core": lambda: lib.tucker_copy_core(None, None),
        "tucker_copy_sv": lambda: lib.tucker_copy_sv(None, None, None),
        "tucker_set_launch_plan": lambda: lib.tucker_set_launch_plan(None, None),
        "tucker_get_launch_plan": lambda: lib.tucker_get_launch_plan(None, None),
        "tucker_profile_enable": lambda: lib.tucker_profile_enable(None, 1),
        "tucker_profile_read": lambda: lib.tucker_profile_read(None, None),
    }
    for name, call in calls.items():
        assert call() == EINVAL, name


def test_batch_entry_points_refuse_null_arguments(lib):
    assert lib.tucker_batch_create(None, None, 0, None) == EINVAL
    assert lib.tucker_batch_update(None, None) == EINVAL
    assert lib.tucker_stream_update_batched(None, None, 0, None) == EINVAL
    assert lib.tucker_stream_update_batched(None, None, 5000, None) == EINVAL
    lib.tucker_batch_kernels.restype = ctypes.c_int64
    assert lib.tucker_batch_kernels(None) == -1
    lib.tucker_batch_destroy(None)         # nothing to do, no crash


def test_queries_on_a_null_state(lib):
    assert lib.tucker_graph_kernels(None) == -1
    for b in (0, 1, 2, 16, 64, 65):
        assert lib.tucker_block_graph_kernels(None, b) == -1
    lib.tucker_last_error.restype = ctypes.c_char_p
    assert lib.tucker_last_error(None) == b"null state"
    lib.tucker_destroy(None)               # nothing to do, no crash
