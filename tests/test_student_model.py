"""The committed trained student (paper_2604_24816_gb300/params/cu_student_trained.json, written by
paper_2604_24816_gb300/distill.py) checked with the FP64 oracle on the CPU: its shape, its stored
training range, and its force error against the teacher on fresh cells near the training distribution.
"""
import json
import os

import numpy as np
import pytest

import nep_inputs as ni
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PATH = os.path.join(ROOT, "paper_2604_24816_gb300", "params", "cu_student_trained.json")
TEACHER = os.path.join(ROOT, "paper_2604_24816_gb300", "params", "cu_nep4_synth.json")


@pytest.fixture(scope="module")
def trained():
    with open(PATH) as f:
        return json.load(f)


def test_trained_student_file(trained):
    for k, v in ni.STUDENT_DIMS.items():
        assert trained[k] == v
    assert len(trained["q_scale"]) == 12 and len(trained["q_lo"]) == 12 and len(trained["q_hi"]) == 12
    assert np.all(np.asarray(trained["q_lo"]) <= np.asarray(trained["q_hi"]))
    tr = trained["training"]
    assert tr["snapshots"] == 2000 and tr["heldout"]["force_rmse"] <= 0.030


def test_trained_student_force_error_vs_teacher(trained):
    """Fresh strained cells with vacancies (0.05 Angstrom displacements): student vs teacher, NEP only."""
    t = oracle.load_model(TEACHER).with_changes(lj_eps=0.0)
    s = oracle.Model(trained).with_changes(lj_eps=0.0)
    d, ref = [], []
    for k in range(3):
        p, b = ni.student_cell(900 + k, (4, 5, 4), 0.05, (0.01, -0.02, 0.0), 2)
        Ft = oracle.energy_forces(t, p, b)[2]
        Fs = oracle.energy_forces(s, p, b)[2]
        d.append(Fs - Ft)
        ref.append(Ft)
    d, ref = np.concatenate(d), np.concatenate(ref)
    rmse = float(np.sqrt(np.mean(d ** 2)))
    assert rmse <= 0.030, rmse
    assert rmse < 0.6 * float(np.sqrt(np.mean(ref ** 2)))
