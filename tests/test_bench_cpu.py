"""Host-side helpers of bench.py: the DRAM traffic read from the committed ncu
summary, and the metric definitions it shares with the oracle (SNR_out of
Section 4.1, the chi^2 bound eps)."""
import math

import numpy as np
import pytest

import bench
from oracle import wproj_oracle as O


def test_profile_traffic_is_read_for_every_reported_kernel():
    for k in ("k_stream_grid", "k_stream_degrid", "k_grid_cells_precision_bf16", "k_grid_cells_precision_f16",
              "k_degrid_precision_bf16", "k_degrid_precision_f16"):
        t = bench.read_profile_traffic(k)
        assert t is not None and t > 1e9, k
    # per entry of G (batched form): a little above the 12 stored bytes
    for k in ("k_grid_cells_batch", "k_degrid_batch"):
        t = bench.read_profile_traffic(k, "traffic_bytes_per_entry")
        assert t is not None and 12.0 <= t <= 16.0, k
    # the figure of a kernel changed since its capture is not used
    assert bench.read_profile_traffic("k_degrid") is None
    # the stream kernels read the stream about once: between 1x and 1.1x the
    # benchmark workload's 40.19 GB stored stream
    for k in ("k_stream_grid", "k_stream_degrid"):
        assert 40.188e9 <= bench.read_profile_traffic(k) <= 1.1 * 40.188e9
    assert bench.read_profile_traffic("no_such_kernel") is None


def test_metric_definitions_agree_with_the_oracle():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((16, 16))
    xr = x + 0.1 * rng.standard_normal((16, 16))
    assert bench.snr_out_db(x, xr) == pytest.approx(O.snr_db(x, xr), rel=1e-12)
    assert bench.synth_eps(0.3, 1000) == pytest.approx(O.epsilon_chi2(0.3, 1000), rel=1e-15)
    assert bench.job_rate(10.5 * 20, 4, 1000.0) == pytest.approx(840.0)
    assert math.isclose(bench.PAIRS_PER_STEP, bench.INNER + 0.5)
