import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MODEL_PATH = os.path.join(ROOT, "paper_2604_24816_gb300", "params", "cu_nep4_synth.json")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the compiled library")


@pytest.fixture(scope="session")
def model():
    import oracle
    return oracle.load_model(MODEL_PATH)


@pytest.fixture(scope="session")
def model_params():
    import json
    with open(MODEL_PATH) as f:
        return json.load(f)
