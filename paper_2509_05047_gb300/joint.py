"""Joint estimation of activity and scatter (Sec. 2.4.2, third scenario).

When the activity is unknown, the paper alternates four steps:
1. reconstruct an activity image with the current scatter estimate;
2. run a short simulation with that activity and the known attenuation image;
3. smooth the new scatter estimate;
4. go back to 1 for a fixed number of iterations.

It starts from a reconstruction without scatter compensation.  The
reconstruction (TOF-OSEM in the paper) is the caller's: `reconstruct`
receives each smoothed estimate and returns the next activity image.  Steps 2
and 3 are the library's calls.  Each iteration replaces the phantom's
activity (`psc_update_activity`, which rebuilds the emission alias table),
zeroes the accumulator, simulates its own range of histories of one seed
(iteration i takes [first + i n, first + (i + 1) n)), and finalizes into the
caller's device buffer.  An iteration's estimate is therefore the one a
single `psc_simulate` + `psc_finalize` on that activity and history range
gives.
"""
from . import (finalize_args, psc_acc_zero, psc_finalize, psc_simulate, psc_update_activity,
               sim_args)


def scatter_iterations(ctx, scanner, phantom, acc, activity0, reconstruct, n_iter, histories, seed,
                       out, lut=0, sens=0, norm=0, sigma=(2.0, 2.0, 2.0), scale=None, first_history=0,
                       stream=None, on_estimate=None):
    """Run n_iter scatter iterations starting from activity0.

    Iteration i runs steps 2 and 3 on the current activity: histories
    [first_history + i histories, first_history + (i + 1) histories) of
    `seed`, then finalize with `sens`, `norm`, `sigma` and `scale` (default
    1 / histories) into `out` (a device float64 tensor of the sinogram's
    shape).  `on_estimate(i, out)` is called after each finalize (for
    example, to copy the estimate out), then `reconstruct(out, i)` returns
    the activity of iteration i + 1 (step 1).  The last reconstruction is
    skipped.  Returns the activity that the last iteration simulated.
    """
    if n_iter < 1 or histories < 1:
        raise ValueError("n_iter and histories must be >= 1")
    sc = 1.0 / histories if scale is None else scale
    fin = finalize_args(acc, sens=sens, norm=norm, sigma=sigma, scale=sc)
    activity = activity0
    for i in range(n_iter):
        psc_update_activity(ctx, phantom, activity)
        psc_acc_zero(ctx, acc, stream)
        psc_simulate(ctx, sim_args(seed, first_history + i * histories, histories, scanner, phantom, acc,
                                   lut=lut), stream=stream)
        psc_finalize(ctx, fin, out, stream)
        if on_estimate is not None:
            on_estimate(i, out)
        if i + 1 < n_iter:
            activity = reconstruct(out, i)
    return activity
