import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))
for _p in (ROOT, TESTS):
    if _p not in sys.path:
        sys.path.insert(0, _p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU runs of the oracle")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def report():
    """Append measured parity figures to $LBM_PARITY_REPORT (a JSON-lines file)
    when that variable is set; a no-op otherwise."""
    import json
    path = os.environ.get("LBM_PARITY_REPORT")

    def rec(name, **values):
        if path:
            with open(path, "a") as f:
                f.write(json.dumps({"test": name, **{k: float(v) for k, v in values.items()}}) + "\n")
    return rec


@pytest.fixture(scope="session")
def oracle_fields(oracle_mod):
    """Fields (phi, u, p) of the FP64 oracle after `steps` steps of a case,
    computed once per session: the parity tests of the float32 and the 16-bit
    storage formats compare against the same oracle runs."""
    cache = {}

    def run(key, case, steps):
        if (key, steps) not in cache:
            p, phi, u, ps = case
            o = oracle_mod.Oracle(p)
            o.init_fields(phi, u, ps)
            o.step(steps)
            cache[(key, steps)] = o.fields()
        return cache[(key, steps)]
    return run
