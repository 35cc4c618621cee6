"""What the trained wake surrogate gains: a two-rotor tandem farm started from
the surrogate's superposed wakes reaches the converged mean hub-plane velocity
in fewer steps than the same farm started from the uniform inflow.  The plain
solver decides: the converged mean is the second half of a long cold
run, and a run counts as settled at the first 1000-step window whose mean is
within twice that run's noise floor of it.

The surrogate is trained in the test on mean wakes of single-rotor runs of this
solver (8 runs, seeded TSR, yaw, U_hub)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_settles_sooner():
    from paper_2402_13171_gb300 import build, inputs as I, lbm, surrogate as S
    build.build()
    X, T, runs = S.generate_wake_data(8, seed=21, shape=(128, 64, 64), D=16.0, spinup=1500, average=1000, every=25)
    net = S.WakeMLP(seed=2)
    net.set_data(X, T)
    loss = net.train(1500, batch=2048, lr=2e-3, seed=3)
    assert loss < 0.01
    nx, ny, nz, D, U = 320, 64, 64, 16.0, 0.05
    rotors = [dict(hub=(32.0, 32.0, 32.0), D=D, tsr=6.0, yaw=0.0, u_hub=U),
              dict(hub=(112.0, 32.0, 32.0), D=D, tsr=6.0, yaw=0.0, u_hub=U)]
    def farm(warm, steps):
        lat = lbm.Lattice.create(nx, ny, nz, nu=1e-3, bc=("inout", "periodic", "freeslip"), seed=5)
        lat.set_inflow(u_ref=(U, 0.0, 0.0), noise_rel=0.01)
        for r in rotors:
            lat.add_turbine(**I.single_turbine(nx, ny, nz, diameter=D, hub=r["hub"], elements_per_blade=16,
                                               tsr=r["tsr"], u_inf=U))
        if warm:
            lat.init_fields(None, S.farm_initial_velocity(net, (nx, ny, nz), rotors, np.full(nz, U), stride=4), None)
        wm = S.WindowMeans(lat, z=32, every=50, window=1000)
        wm.advance(steps)
        lat.destroy()
        return wm

    cold = farm(False, 30000)
    ref, noise = S.converged_reference(cold, 15000)
    warm = farm(True, 12000)
    tol = 2.0 * noise
    t_cold, t_warm = S.settle_step(cold, ref, tol), S.settle_step(warm, ref, tol)
    print(f"noise floor {noise:.3e}; settled (window mean within {tol:.3e} of the converged mean): "
          f"cold {t_cold}, warm {t_warm}; surrogate loss {loss:.2e}")
    print("cold errors", np.round(S.window_errors(cold, ref)[:12], 4))
    print("warm errors", np.round(S.window_errors(warm, ref)[:12], 4))
    assert t_warm is not None and t_cold is not None and t_warm < t_cold
    net.destroy()
