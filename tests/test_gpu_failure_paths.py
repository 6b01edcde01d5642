"""Failure paths of the C ABI on the GPU, each made on the host without faulting
the GPU: invalid parameters are rejected before any work is queued
(LSB_EINVAL), a non-finite state is detected by the observables reduction
(LSB_EUNSTABLE: a NaN acceleration handed over as a parameter, and a run driven
unstable), a device work list that overflows is reported (LSB_ENOMEM: a level
set with a sign change at every cell has more interface cells and cut links
than the lists hold), and a bounded device-side wait that runs out ends its
kernel and is reported (LSB_ETIMEOUT: the persistent level-set launch with a
wait limit of zero).  After each error the CUDA context stays usable: a new
handle on the same device runs and matches a handle that never saw an error.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EINVAL, ENOMEM, EUNSTABLE, ETIMEOUT = 1, 2, 4, 5


def _channel(n=(64, 32), nu=0.1, force=1e-6):
    D = len(n)
    return dict(lattice="D2Q9", base=n, block=(32, 8), periodic=(True, False), rho_phys=(1.0, 1.0),
                nu=(nu, nu), body_force=(force, 0.0), phi0=-np.ones(int(np.prod(n))), n_ext=0,
                reinit_every=0, ls_active=False)


def _bubble(N=48, seed=3):
    rng = np.random.default_rng(seed)
    x = np.arange(N) + 0.5
    X, Y = np.meshgrid(x, x)
    xc, yc = N / 2 + rng.random(), N / 2 + rng.random()
    phi = 8.0 - np.sqrt((X - xc) ** 2 + (Y - yc) ** 2)
    return dict(lattice="D2Q9", base=(N, N), block=(32, 8), periodic=(False, False), rho_phys=(1.0, 0.1),
                nu=(0.1, 0.1), sigma=1e-3, gravity=(0.0, -1e-5), x_ref=(xc, yc), phi0=phi.reshape(-1))


def _context_still_usable():
    from paper_2601_05936_gb300 import lsb
    a = lsb.Grid(_channel())
    a.step(5)
    u = a.get("u")
    assert np.isfinite(u).all() and np.abs(u).max() > 0
    a.close()


@pytest.mark.parametrize("bad", [dict(nu=(0.1, 0.0)), dict(nu=(0.1, -1.0)), dict(rho_phys=(1.0, float("nan"))),
                                 dict(sigma=float("nan")), dict(sigma=-1e-3), dict(n_ext=-1)],
                         ids=["nu_zero", "nu_negative", "rho_nan", "sigma_nan", "sigma_negative", "n_ext_negative"])
def test_invalid_parameters_are_rejected(bad):
    from paper_2601_05936_gb300 import lsb
    with pytest.raises(lsb.LsbError) as e:
        lsb.Grid(dict(_channel(), **bad))
    assert e.value.status == EINVAL
    g = lsb.Grid(_channel())
    with pytest.raises(lsb.LsbError) as e:
        g.set_params(dict(_channel(), **bad))
    assert e.value.status == EINVAL
    g.step(2)  # the rejected call changed nothing
    ref = lsb.Grid(_channel())
    ref.step(2)
    assert np.array_equal(g.get("f"), ref.get("f"))
    g.close()
    ref.close()


def test_nan_parameter_is_reported_unstable():
    """A NaN acceleration set on the host reaches the populations; the next synchronising
    call reports the non-finite state."""
    from paper_2601_05936_gb300 import lsb
    case = dict(_bubble(), ls_active=False)  # the interface stays put: the NaN stays in the populations
    g = lsb.Grid(case)
    g.step(2)
    assert g.observables()[0]["mass"].sum() > 0
    g.set_params(dict(case, gravity=(0.0, float("nan"))))
    g.step(2)
    with pytest.raises(lsb.LsbError) as e:
        g.observables()
    assert e.value.status == EUNSTABLE
    with pytest.raises(lsb.LsbError) as e:  # the error stays latched on the handle
        g.sync()
    assert e.value.status == EUNSTABLE
    g.close()
    _context_still_usable()


def test_divergent_run_is_reported_unstable():
    """A static drop at density ratio 1000 with the liquid viscosity at 0.02, below the
    stability limit of the explicit normal-stress coupling (the FP64 oracle's state
    overflows after ~500 steps with the interface held fixed): the run is stepped until
    the observables report the non-finite state."""
    from paper_2601_05936_gb300 import lsb, workloads
    case = workloads.static_drop(n=48, levels=1, radius_base=10.0, nu_l=0.02)
    case.update(ls_active=False, n_ext=0, reinit_every=0)
    g = lsb.Grid(case)
    with pytest.raises(lsb.LsbError) as e:
        for _ in range(60):
            g.step(50)
            g.observables()
    assert e.value.status == EUNSTABLE
    g.close()
    _context_still_usable()


def test_work_list_overflow_is_reported():
    """A sign change at every cell of a 1024 x 1024 level: ~1 M interface cells and ~4 M
    cut links against lists of 262 144 cells and 2 M links.  Every list write past the
    end is skipped on the device and the overflow is latched."""
    from paper_2601_05936_gb300 import lsb
    n = 1024
    rng = np.random.default_rng(41)
    phi = np.where(rng.random(n * n) < 0.5, -0.5, 0.5)
    case = dict(lattice="D2Q9", base=(n, n), block=(32, 8), periodic=(True, True), rho_phys=(1.0, 0.1),
                nu=(0.1, 0.1), sigma=0.0, phi0=phi, ls_active=False, n_ext=0, reinit_every=0)
    with pytest.raises(lsb.LsbError) as e:
        g = lsb.Grid(case)
        g.sync()
    assert e.value.status == ENOMEM
    _context_still_usable()


def test_persistent_barrier_timeout_is_reported():
    """The persistent level-set launch (one cooperative kernel with a grid barrier between
    passes) with a wait limit of zero: every CTA that has to wait gives up at once and
    leaves the kernel, and the next synchronising call reports the timeout.  The same
    handle with the default limit, created afresh, matches the per-pass launches."""
    from paper_2601_05936_gb300 import lsb
    g = lsb.Grid(_bubble())
    g.set_driver(1)
    g.set_wait_limit(0)
    g.step(1)
    with pytest.raises(lsb.LsbError) as e:
        g.sync()
    assert e.value.status == ETIMEOUT
    g.close()
    ok = lsb.Grid(_bubble())
    ok.set_driver(1)
    ok.step(3)
    ok.sync()
    ref = lsb.Grid(_bubble())
    ref.step(3)
    assert np.array_equal(ok.get("phi"), ref.get("phi"))
    assert np.array_equal(ok.get("u"), ref.get("u"))
    with pytest.raises(lsb.LsbError) as e:
        ok.set_wait_limit(-1)
    assert e.value.status == EINVAL
    ok.close()
    ref.close()
