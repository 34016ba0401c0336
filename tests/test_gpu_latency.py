"""The device latency probe behind the sweeps' latency bound (lsq_measure_latency)."""
import pytest

pytestmark = pytest.mark.gpu


def test_latency_probe_values_are_plausible(lsq):
    """Four bounded probes, each a positive time in a physically sensible range: a dependent
    L2 load and a DSMEM load take tens to hundreds of ns, a cluster barrier a few hundred, a
    round trip between two SMs through global memory under tens of microseconds."""
    lat = lsq.measure_latency()
    assert 20.0 < lat["l2_load_ns"] < 5000.0, lat
    assert 20.0 < lat["dsmem_load_ns"] < 5000.0, lat
    assert 20.0 < lat["cluster_barrier_ns"] < 20000.0, lat
    assert 50.0 < lat["sm_round_trip_ns"] < 50000.0, lat
    assert 50.0 < lat["sm_round_trip_fenced_ns"] < 50000.0, lat
    # a value handed between SMs through memory costs at least one L2 access each way
    assert lat["sm_round_trip_ns"] > lat["l2_load_ns"]
