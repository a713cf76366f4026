import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU checks")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def genome29():
    """The 29x overlap workload (4.6 Mbp genome, about 314k pairs), built
    once per session for every test that uses it."""
    from paper_2309_07270_gb300 import workloads as W
    return W.genome_overlaps()


@pytest.fixture(scope="session")
def oracle_full(orc):
    """Oracle results and per-extension cell counts of whole workloads,
    computed once per session on every host core and kept by key."""
    cache = {}

    def get(key, w):
        if key not in cache:
            cache[key] = orc.align_pairs(w.packed, w.read_off, w.read_len, w.pairs, w.match,
                                         w.mismatch, w.gap, w.x, nthreads=os.cpu_count() or 1,
                                         with_cells=True)
        return cache[key]
    return get
