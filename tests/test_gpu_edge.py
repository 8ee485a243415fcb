"""Degenerate runs and rejected configurations through the C ABI (GPU).

* Every particle killed: a SEIR report larger than the human population has
  probability 0 under every particle (Listing 2's observation is
  Binomial(z, rho) with z at most 7,370), so the normaliser finds no weight at
  that checkpoint.  The run stops there with SMC_EDEGENERATE and log Z = -inf,
  after as many segments as the oracle, whose other outputs it matches.
* Configurations outside the header's ranges (N < 1 or above
  SMC_MAX_PARTICLES, max_segments outside 0..2^24, a negative or non-finite
  ESS threshold) return SMC_EINVAL before any device work.
"""
import math

import numpy as np
import pytest

import inputs
import oracle
from parity import assert_parity_fp64, run_pair

pytestmark = pytest.mark.gpu

KILLING_REPORTS = [[1e5], [-1.0, 1e5], [-1.0, -1.0, 3.0, 1e5, -1.0]]


@pytest.mark.parametrize("y", KILLING_REPORTS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_seir_every_particle_killed(y, precision):
    from paper_2112_00364_gb300 import smc

    g, o = run_pair("seir", 1000, seed=3, precision=precision, obs=np.array(y))
    assert o["status"] == oracle.EDEGENERATE and g["status"] == smc.EDEGENERATE
    assert g["log_z_value"] == -math.inf
    assert g["n_segments"] == o["n_segments"] == y.index(1e5) + 1
    assert g["n_resamples"] == o["n_resamples"]
    assert not np.isfinite(g["final_logw"]).any()
    if precision == "fp64":
        assert_parity_fp64(g, o)


@pytest.mark.parametrize("kw", [dict(max_segments=-1), dict(max_segments=(1 << 24) + 1),
                                dict(ess_threshold=-0.5), dict(ess_threshold=math.nan),
                                dict(ess_threshold=math.inf)])
def test_run_rejects_bad_configurations(kw):
    from paper_2112_00364_gb300 import smc

    m = smc.Model("lg", obs=inputs.lg_observations(5, seed=1))
    try:
        with pytest.raises(smc.SmcError) as e:
            smc.run(m, 100, 1, **kw)
        assert e.value.status == smc.EINVAL
    finally:
        m.close()


@pytest.mark.parametrize("N", [0, -5, None])
def test_particle_count_outside_range(N):
    # checked through smc_workspace_bytes, which validates the same run
    # configuration and allocates nothing (a run would first allocate its
    # outputs)
    from paper_2112_00364_gb300 import smc

    N = smc.MAX_PARTICLES + 1 if N is None else N
    m = smc.Model("lg", obs=inputs.lg_observations(5, seed=1))
    try:
        with pytest.raises(smc.SmcError) as e:
            m.workspace_bytes(N)
        assert e.value.status == smc.EINVAL
        assert m.workspace_bytes(smc.MAX_PARTICLES) > 40 * smc.MAX_PARTICLES
    finally:
        m.close()
