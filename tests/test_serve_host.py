"""Host-side pieces of the server (no GPU): latency statistics."""
from paper_2112_10223_gb300.serve import ServeStats


def test_percentiles_and_summary():
    st = ServeStats(requests=5, batches=2, seconds=2.0, nnz_in=100, latencies=[0.5, 0.1, 0.4, 0.2, 0.3])
    assert st.pct(50) == 0.3
    assert st.pct(99) == 0.5
    assert st.pct(0) == 0.1
    s = st.summary()
    assert s["nnz_per_s"] == 50 and s["requests_per_s"] == 2.5 and s["mean_batch"] == 2.5
    assert abs(s["p50_ms"] - 300.0) < 1e-9 and abs(s["max_ms"] - 500.0) < 1e-9
