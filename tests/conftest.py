import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# test modules whose oracle references are computed by tests/oracle_jobs.py
ORACLE_JOB_MODULES = ('test_gpu_parity_128.py',)


def pytest_configure(config):
    config.addinivalue_line('markers', 'gpu: needs a CUDA GPU (GB300, sm_103a)')
    config.addinivalue_line('markers', 'slow: CPU test that takes more than a few seconds')


def pytest_collection_finish(session):
    """Start the long oracle reference jobs as soon as the session knows it
    will run their tests on a GPU, so they overlap the rest of the suite."""
    if session.config.option.collectonly:
        return
    wanted = any(os.path.basename(str(item.fspath)) in ORACLE_JOB_MODULES
                 for item in session.items)
    if not wanted:
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except ImportError:
        return
    import oracle_jobs
    oracle_jobs.start()


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get('oracle_jobs')
    if mod is not None:
        mod.shutdown()
