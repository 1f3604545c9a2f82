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


STUDENT_SEED = 7331


@pytest.fixture(scope="session")
def student_params():
    """A seeded, untrained model of the student shape (n_max 3/3, l_max 2, no 4-body, 16 neurons)."""
    import nep_inputs as ni
    from oracle.write_model import make_model
    return make_model(ni.STUDENT_DIMS, STUDENT_SEED)


@pytest.fixture(scope="session")
def student_model(student_params):
    import oracle
    return oracle.Model(student_params)


@pytest.fixture(scope="session")
def trained_student_params():
    import json
    with open(os.path.join(ROOT, "paper_2604_24816_gb300", "params", "cu_student_trained.json")) as f:
        return json.load(f)
