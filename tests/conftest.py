import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built liblsq.so")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if gpu_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def orc():
    pkg = os.environ.get("LSQ_ORACLE_PKG")
    if pkg:
        # a copy of the oracle package with one planted mistake in its Python layer
        # (tests/test_oracle_mutants.py): the pins run against it and must fail
        import importlib.util
        here = os.path.join(pkg, "oracle")
        spec = importlib.util.spec_from_file_location("oracle", os.path.join(here, "__init__.py"),
                                                      submodule_search_locations=[here])
        mod = importlib.util.module_from_spec(spec)
        sys.modules["oracle"] = mod
        spec.loader.exec_module(mod)
        mod.build()
        return mod
    import oracle
    mutant = os.environ.get("LSQ_ORACLE_MUTANT")
    if mutant:
        # a copy of the oracle with one planted mistake (tests/test_oracle_mutants.py):
        # the pins run against it and must fail
        oracle.build = lambda force=False: mutant
    else:
        oracle.build()
    return oracle


@pytest.fixture(scope="session")
def lsq():
    """The CUDA package, built in-tree; a GPU test fails loudly if it cannot load."""
    import paper_1806_02968_gb300 as pkg
    pkg.build()
    from paper_1806_02968_gb300 import api
    api.L.load()
    return api
