"""Reader for the worked-example fixtures in tests/golden (one fact per line)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    facts = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            facts.setdefault(key, []).append(vals)
    return facts


def dfa_from(facts):
    """(num_states, symbols string, delta int32 [Q, S] with -1 for q_e, q0, finals)."""
    Q = int(facts["states"][0][0])
    syms = facts["symbols"][0][0]
    delta = np.full((Q, len(syms)), -1, dtype=np.int32)
    for src, a, dst in facts.get("edge", []):
        delta[int(src), syms.index(a)] = int(dst)
    q0 = int(facts["start"][0][0])
    finals = [int(x) for x in facts["final"][0]]
    return Q, syms, delta, q0, finals


def symbol_map(syms):
    m = np.full(256, 0xFF, dtype=np.uint8)
    for i, ch in enumerate(syms):
        m[ord(ch)] = i
    return m


def state(tok, Q):
    return Q if tok == "qe" else int(tok)
