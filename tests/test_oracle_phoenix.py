"""The Phoenix Argmax baseline (SecPE Sec. 3.2), in the oracle: m = C' - 1
comparisons s = sum_i Sign(y - RotL(y, i)), then one more Sign; its op
counts follow the paper's m + 1 Signs and m + 1 rotations, its plaintext
pipeline returns the exact argmax, and the encrypted circuit decodes to the
plaintext pipeline within 2^-12 with the exact index."""
import json
import os

import numpy as np
import pytest

from oracle import plainsim
from paper_2502_00847_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


def test_phoenix_plaintext_pipeline_exact_index():
    for C in (2, 3, 4, 6, 14):
        for s in range(20):
            q = workloads.toy_query(seed=500 + s, K=3, C=C)
            z = plainsim.ensemble_phoenix_argmax(q.logits, q.d_min, q.d_max, 2048)
            assert int(np.argmax(z)) == int(np.argmax(q.logits.mean(0)))
    for q in workloads.argmax_queries(64, seed=4):
        z = plainsim.ensemble_phoenix_argmax(q.logits, q.d_min, q.d_max, 32768)
        assert int(np.argmax(z)) == int(np.argmax(q.logits.mean(0)))


@pytest.mark.parametrize("C,K,seed", [(2, 3, 1), (4, 2, 2), (3, 3, 3)])
def test_oracle_phoenix_decodes_to_plaintext_pipeline(toy_oracle, C, K, seed):
    o = toy_oracle
    facts = json.load(open(GOLDEN))["phoenix_op_counts"]
    q = workloads.toy_query(seed=seed, K=K, C=C)
    cts = [o.encrypt_logits(q.logits[i], C, q.d_min, seed=q.enc_seeds[i]) for i in range(K)]
    y = o.aggregate(cts, q.d_min, q.d_max)
    o.reset_counters()
    z = o.phoenix_argmax(y, C, q.qseed)
    m = (1 << (C - 1).bit_length()) - 1
    assert facts["sign_calls"] == facts["rotations"] == "m + 1"
    assert o.counters["signs"] == m + 1 and o.counters["rotations"] == m + 1
    zd = o.decrypt(z, C)
    zp = plainsim.ensemble_phoenix_argmax(q.logits, q.d_min, q.d_max, o.n // 2)
    assert np.max(np.abs(zd - zp)) < 2.0 ** -12
    assert int(np.argmax(zd)) == int(np.argmax(q.logits.mean(0)))
