"""Host-side validation of tucker_init_sthosvd's configuration (through the C ABI, no GPU): every
rule rejects a bad value with TUCKER_EINVAL and its message before any device work, so a caller
learns of a wrong capacity, size or tolerance at once instead of from a latched device error."""

import ctypes
import math

import pytest

EINVAL = 1
DUMMY = 0x1000   # never dereferenced: validation returns before the data pointer is used


@pytest.fixture(scope="module")
def pkg():
    from paper_2308_16395_gb300 import build as b

    b.build()
    import paper_2308_16395_gb300 as p

    p.load_library()
    return p


def _init(pkg, cfg, n_init=4):
    lib = pkg.load_library()
    h = ctypes.c_void_p(12345)
    rc = lib.tucker_init_sthosvd(ctypes.byref(cfg), ctypes.c_void_p(DUMMY), int(n_init),
                                 ctypes.c_void_p(0), ctypes.byref(h))
    return rc, h.value


def _cfg(pkg, **kw):
    base = dict(n=(24, 20, 16), tau=1e-3)
    base.update(kw)
    n, tau = base.pop("n"), base.pop("tau")
    return pkg.make_config(n, tau, **base)


@pytest.mark.parametrize("change,message", [
    (dict(tau=0.0), "tau must be > 0"),
    (dict(tau=-1e-3), "tau must be > 0"),
    (dict(tau=math.inf), "tau must be > 0"),
    (dict(tau=math.nan), "tau must be > 0"),
    (dict(n=(24, 20, 513)), "n_3 must be in 1..512"),
    (dict(n=(24, 0, 16)), "n_2 must be in 1..512"),
    (dict(rank_cap=[25, 0, 0, 0]), "rank_cap[0] must be in 0..n_1"),
    (dict(rank_cap=[0, 0, 0, 513]), "streaming rank cap must be <= 512"),
    (dict(precision="fp64", n=(300, 20, 16)), "above 256 for this precision"),
    (dict(steps_cap=2), "steps_cap must be >= n_init"),
    (dict(core_cap=-1), "core_cap must be >= 0"),
    (dict(block_cap=65), "block_cap must be in 0..64"),
    (dict(block_cap=-1), "block_cap must be in 0..64"),
])
def test_bad_configuration_is_refused_before_device_work(pkg, capfd, change, message):
    rc, h = _init(pkg, _cfg(pkg, **change))
    assert rc == EINVAL
    assert h is None                       # *out is cleared on every failure
    assert message in capfd.readouterr().err


@pytest.mark.parametrize("n_init", [0, -3, 513])
def test_n_init_out_of_range_is_refused(pkg, capfd, n_init):
    rc, h = _init(pkg, _cfg(pkg), n_init=n_init)
    assert rc == EINVAL and h is None
    assert "n_init must be in 1..512" in capfd.readouterr().err


def test_dimension_and_type_checks(pkg, capfd):
    c = _cfg(pkg)
    c.ndim = 9
    assert _init(pkg, c)[0] == EINVAL
    c = _cfg(pkg)
    c.dtype = 7
    assert _init(pkg, c)[0] == EINVAL
    c = _cfg(pkg)
    c.precision = 3
    assert _init(pkg, c)[0] == EINVAL
    err = capfd.readouterr().err
    assert "ndim must be in 2..8" in err and "bad dtype" in err and "bad precision" in err


def test_null_arguments(pkg):
    lib = pkg.load_library()
    h = ctypes.c_void_p()
    assert lib.tucker_init_sthosvd(None, ctypes.c_void_p(DUMMY), 4, None, ctypes.byref(h)) == EINVAL
    cfg = _cfg(pkg)
    assert lib.tucker_init_sthosvd(ctypes.byref(cfg), None, 4, None, ctypes.byref(h)) == EINVAL
    assert lib.tucker_init_sthosvd(ctypes.byref(cfg), ctypes.c_void_p(DUMMY), 4, None, None) == EINVAL
