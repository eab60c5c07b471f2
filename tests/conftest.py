"""Shared pytest configuration.

Markers:
  gpu  -- needs a CUDA device and the in-tree CUDA library (run with -m gpu).
Tests without the marker run on any host (-m "not gpu").
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the in-tree CUDA library")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build()
    return oracle


def make_oracle(params: dict):
    """Oracle domain from a workload parameter dict (nx, ny, nz, dx + the rest)."""
    from oracle.oracle import Oracle
    p = dict(params)
    nx, ny, nz, dx = p.pop("nx"), p.pop("ny"), p.pop("nz"), p.pop("dx")
    return Oracle(nx, ny, nz, dx, **p)
