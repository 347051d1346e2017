"""CPU checks of DFA groups (several DFAs on one input, Sec. 5): the joint
classes the library builds equal the common refinement of the DFAs' alphabet
classes, computed here from the specs' delta columns; the group's limits are
enforced; a group of host-only DFAs has no device image.  No CUDA call is made
(dfa_create_host does none, and a host-only group makes none)."""
import numpy as np
import pytest

import gen
import oracle


@pytest.fixture(scope="module")
def dm():
    from paper_1210_5093_gb300 import build
    build.build()
    import paper_1210_5093_gb300 as dm
    dm.lib()
    return dm


def _column_key(spec, b):
    """Behaviour of byte b in one DFA: None outside Sigma, else its delta column."""
    sym = spec.symbol_of_byte()[b]
    if sym < 0:
        return None
    d = np.asarray(spec.delta, dtype=np.int64).reshape(spec.num_states, spec.num_symbols)
    return tuple(d[:, sym].tolist())


def _refinement(specs):
    """Partition of the 256 bytes: b ~ b' iff they behave alike in every DFA."""
    keys = [tuple(_column_key(s, b) for s in specs) for b in range(256)]
    ids = {}
    return np.array([ids.setdefault(k, len(ids)) for k in keys]), len(ids)


def _same_partition(a, b):
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


def _protein(seed, Q):
    return gen.class_dfa(seed, Q, 20, 0.02, 0.35, max(1, Q // 100), "protein")


def test_joint_classes_of_protein_dfas(dm):
    specs = [_protein(10 + i, q) for i, q in enumerate((12, 40, 200))]
    g = dm.Group([dm.Dfa.from_spec(s, host_only=True) for s in specs])
    want, J = _refinement(specs)
    got = g.joint_classes()
    assert _same_partition(got, want)
    info = g.info()
    assert info.num_dfas == 3 and info.joint_classes == J == 21  # 20 letters + outside Sigma
    assert info.state_bytes == 1 and info.max_states_ext == 201
    assert info.device_bytes == 0
    # one row per joint class plus the identity row, for every DFA
    need = sum((J + 1) * (s.num_states + 1) for s in specs)
    assert need <= info.table_bytes <= need + 3 * (J + 1) * 15
    # sum of the largest sets (Eq. 12; the start set {q0} counts 1)
    imax = [oracle.Dfa.from_spec(s).isets()[1] for s in specs]
    assert info.sum_max_set == sum(max(1, m) for m in imax)


def test_joint_classes_of_unrelated_dfas(dm):
    """A byte-classed DFA and a protein DFA: the refinement pairs their classes."""
    specs = [gen.class_dfa(5, 30, 6, 0.05, 0.4, 2, "byte"), _protein(6, 300)]
    g = dm.Group([dm.Dfa.from_spec(s, host_only=True) for s in specs])
    want, J = _refinement(specs)
    assert _same_partition(g.joint_classes(), want)
    assert g.info().joint_classes == J and J > 21
    assert g.info().state_bytes == 2
    # a single DFA's joint classes are its own classes
    one = dm.Group([dm.Dfa.from_spec(specs[0], host_only=True)])
    d = dm.Dfa.from_spec(specs[0], host_only=True)
    assert _same_partition(one.joint_classes(), d.class_of_bytes().astype(np.int64))


def test_group_limits(dm):
    small = [dm.Dfa.from_spec(_protein(20 + i, 10), host_only=True) for i in range(17)]
    dm.Group(small[:16])
    with pytest.raises(dm.DfaError) as e:                       # more than 16 DFAs
        dm.Group(small)
    assert e.value.status == dm.EINVAL
    with pytest.raises(dm.DfaError) as e:                       # none
        dm.Group([])
    assert e.value.status == dm.EINVAL
    big = dm.Dfa.from_spec(gen.random_dfa(3, 4096, 2, num_finals=2, byte_to_symbol=_ab()),
                           host_only=True)
    with pytest.raises(dm.DfaError) as e:                       # |Q| + 1 > 4096
        dm.Group([big])
    assert e.value.status == dm.EINVAL
    plain = dm.Dfa.from_spec(gen.plain_dfa(1), host_only=True)   # 256 classes: 256 joint classes
    with pytest.raises(dm.DfaError) as e:
        dm.Group([plain])
    assert e.value.status == dm.EINVAL
    wide = [dm.Dfa.from_spec(_protein(30 + i, 2000), host_only=True) for i in range(2)]
    with pytest.raises(dm.DfaError) as e:                       # joint tables above 160 KiB
        dm.Group(wide)
    assert e.value.status == dm.EINVAL
    # sets: three 4000-state permutation DFAs over one symbol (I = Q each)
    perm = []
    for i in range(3):
        d = np.roll(np.arange(4000, dtype=np.int32), 1 + i).reshape(4000, 1)
        perm.append(dm.Dfa(4000, 1, d, 0, [1], byte_to_symbol=_one_symbol(), host_only=True))
    dm.Group(perm[:2])
    with pytest.raises(dm.DfaError) as e:                       # sum of largest sets above 8192
        dm.Group(perm)
    assert e.value.status == dm.EINVAL


def _ab():
    m = np.full(256, 0xFF, dtype=np.uint8)
    m[ord("a")], m[ord("b")] = 0, 1
    return m


def _one_symbol():
    m = np.full(256, 0xFF, dtype=np.uint8)
    m[ord("a")] = 0
    return m


def test_host_only_group_has_no_device_image(dm):
    g = dm.Group([dm.Dfa.from_spec(_protein(40, 50), host_only=True)])
    with pytest.raises(dm.DfaError) as e:
        g.plan_chunks(1 << 20)
    assert e.value.status == dm.EHOSTONLY
    with pytest.raises(dm.DfaError) as e:
        g.workspace_size(1 << 20)
    assert e.value.status == dm.EHOSTONLY
