"""Host-side logic of bench.py that needs no GPU: the oracle baseline spread
over host cores (one spawned process per core)."""
import importlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    # imported by name, so that the spawned workers find the same functions
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_oracle_pool_runs_one_sample_per_process():
    bench = load_bench()
    one_t, one_u, _ = bench.oracle_sample(n_side=4, n_time=1)
    pool = bench.OraclePool(cores=2)
    try:
        wall, units, sample = pool.run(n_side=4, n_time=1)
    finally:
        pool.close()
    assert wall > 0
    # two independent copies of the same deterministic sample
    assert units == 2 * one_u[0]
    assert sample.startswith("2 processes")
