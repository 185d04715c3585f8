"""The entry point's smoke run (one small forward, backward and Metropolis
pass of the Be-shaped system on cuda:0, the first two checked against the
oracle) passes."""

import os
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_smoke_entry_point(lib):
    sys.path.insert(0, ROOT)
    import __graft_entry__

    __graft_entry__.smoke()
