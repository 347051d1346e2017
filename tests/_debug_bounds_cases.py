"""Parity cases run against the debug build of the library (libdfamatch_debug.so,
loaded when DFA_DEBUG_BOUNDS=1): the same kernels with every state, class, set
slot and chunk bound checked before use.  A failed check would surface as
DFA_EBOUNDS in a result; every answer must instead equal the oracle's.
Run as a script in its own process (the library is chosen at load time)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import gen      # noqa: E402
import oracle   # noqa: E402


def main():
    assert os.environ.get("DFA_DEBUG_BOUNDS") == "1"
    import torch
    import paper_1210_5093_gb300 as dm
    assert dm.LIB_PATH.endswith("libdfamatch_debug.so"), dm.LIB_PATH
    checked = 0

    def check(d, spec, data, **kw):
        nonlocal checked
        st, fs, acc = d.match(data, **kw)
        host = data.cpu().numpy() if isinstance(data, torch.Tensor) else data
        want = oracle.Dfa.from_spec(spec).run(host)
        assert st != dm.EBOUNDS, ("bounds check failed", spec.name, kw)
        assert (st, fs, acc) == want or (st == want[0] != 0), (spec.name, kw, (st, fs, acc), want)
        checked += 1

    m3 = np.full(256, 0xFF, dtype=np.uint8)
    m3[:3] = np.arange(3)
    cases = [
        (gen.plain_dfa(1), gen.uniform_bytes(1, 1 << 20), [{}, {"num_chunks": 1024}]),
        (gen.random_dfa(2, 5, 3, missing=0.2, byte_to_symbol=m3),
         (gen.uniform_bytes(3, 300_000) % 3).astype(np.uint8),
         [{}, {"num_chunks": 17}, {"lookahead": 0}, {"lookahead": 3}, {"boundary_window": 64}]),
        (gen.random_dfa(4, 300, 256, num_finals=30, missing=0.02), gen.uniform_bytes(5, 2 << 20),
         [{}, {"num_chunks": 3000}, {"lookahead": 2}]),
        (gen.regex_dfa(2), gen.zipf_text(2, 16 << 20),
         [{}, {"lookahead": 2}, {"lookahead": 4}, {"lookahead": 0}, {"boundary_window": 256},
          {"num_chunks": 5000, "multiplicity": 3}]),
        (gen.protein_dfa(3), gen.protein_text(3, 16 << 20), [{}, {"boundary_window": 256}]),
        (gen.class_dfa(81, 1288, 256, 0.02, 0.3, 12, "byte"), gen.zipf_text(83, 4 << 20),
         [{}, {"lookahead": 2}]),                                      # table read through L2
        (gen.class_dfa(1020, 20000, 20, 0.2, 0.9, 200, "protein"), gen.protein_text(9, 300_000),
         [{}, {"lookahead": 0, "num_chunks": 40}]),                    # multi-pass chunks
    ]
    for spec, data, kws in cases:
        d = dm.Dfa.from_spec(spec)
        print("case", spec.name, len(data), flush=True)
        for kw in kws:
            check(d, spec, data, **kw)
            check(d, spec, data[: len(data) // 3 + 7], **kw)
        if spec.byte_to_symbol is not None and (spec.byte_to_symbol == 0xFF).any():
            bad = data.copy()       # a byte outside Sigma in the middle: DFA_ESYMBOL
            bad[len(bad) // 2] = int(np.nonzero(spec.byte_to_symbol == 0xFF)[0][0])
            check(d, spec, bad)
    # a batch of several DFAs (shared-memory and L2 tables), with graph replay
    specs = [gen.regex_dfa(2), gen.plain_dfa(1), gen.class_dfa(81, 1288, 256, 0.02, 0.3, 12, "byte")]
    dfas = [dm.Dfa.from_spec(s) for s in specs]
    xs = [gen.zipf_text(40 + i, 50_000 * (i + 1) + i) for i in range(9)]
    tens = [torch.from_numpy(x).cuda() for x in xs]
    picks = [i % 3 for i in range(9)]
    b = dm.Batch([dfas[p] for p in picks], tens)
    out = torch.zeros(12 * len(tens), dtype=torch.uint8, device="cuda")
    for graph in (False, True):
        b.launch(out, graph=graph)
        torch.cuda.synchronize()
        for i, (fs, acc, st) in enumerate(dm.results_from(out)):
            assert st != dm.EBOUNDS
            assert (st, fs, acc) == oracle.Dfa.from_spec(specs[picks[i]]).run(xs[i])
            checked += 1
    b.close()
    # the pipelined host path (map tests and their combine), on pinned memory
    w = gen.regex_workload(2, 96 << 20)
    d = dm.Dfa.from_spec(w.spec)
    d.set_tuning(host_segment_bytes=8 << 20)
    check(d, w.spec, torch.from_numpy(w.data).pin_memory())
    # random DFAs with random launch options (as the random-options parity test)
    for case in range(20):
        u = gen.unit(gen.draws(gen.key(7000 + case, 3), 32))
        Q, S = 1 + int(u[0] ** 2 * 700), 1 + int(u[1] * 40)
        m = np.full(256, 0xFF, dtype=np.uint8)
        alphabet = gen.permutation(gen.key(7000 + case, 4), 256)[: S + int(u[2] * 3 * S)]
        m[alphabet] = np.arange(len(alphabet)) % S
        spec = gen.random_dfa(7100 + case, Q, S, num_finals=max(1, Q // 3),
                              missing=0.15 * u[3], byte_to_symbol=m)
        d = dm.Dfa.from_spec(spec)
        n = int(u[4] ** 2 * 400_000)
        x = alphabet[gen.below(gen.draws(gen.key(7200 + case, 5), n), len(alphabet))].astype(np.uint8)
        for trial in range(3):
            v = gen.unit(gen.draws(gen.key(7300 + case, 6 + trial), 8))
            kw = {"num_chunks": 0 if v[0] < 0.4 else 1 + int(v[1] ** 2 * 5000),
                  "lookahead": int(v[2] * 5)}
            if kw["lookahead"] >= 1 and v[3] < 0.3:
                kw["boundary_window"] = [1, 16, 256, 4096][int(v[4] * 4)]
            check(d, spec, x, **kw)
    # groups of DFAs sharing one stage: protein DFAs at several K and chunk
    # counts, and a group whose byte-classed DFA has every byte in Sigma while
    # its protein DFA does not (a byte outside the letters fails only the latter)
    groups = [(gen.protein_group_dfas(7), gen.protein_text(11, 4 << 20)),
              ([gen.class_dfa(75, 60, 8, 0.05, 0.4, 2, "byte")] + gen.protein_group_dfas(8, (20, 90)),
               gen.protein_text(12, 1 << 20))]
    groups[1][1][300_000] = ord("#")
    for gspecs, x in groups:
        g = dm.Group([dm.Dfa.from_spec(s) for s in gspecs])
        dev = torch.from_numpy(x).cuda()
        want = [oracle.Dfa.from_spec(s).run(x) for s in gspecs]
        for kw in ({}, {"states_per_thread": 1}, {"states_per_thread": 16, "num_chunks": 3000},
                   {"num_chunks": 7}):
            got = g.match(dev, **kw)       # raises on DFA_EBOUNDS
            assert got == want, (kw, got, want)
            checked += len(gspecs)
        g.close()
    # a group on host input of 40 MiB: segments copied while earlier ones are
    # matched (continuation launches publishing state maps, Eq. 8 over them)
    gspecs = gen.protein_group_dfas(7, (16, 100, 480))
    g = dm.Group([dm.Dfa.from_spec(s) for s in gspecs])
    x = gen.protein_text(13, 40 << 20)
    x[(16 << 20) - 1] = ord("#")       # the lookahead byte of the second segment
    want = [oracle.Dfa.from_spec(s).run(x) for s in gspecs]
    assert g.match(x) == want
    x[(16 << 20) - 1] = ord("A")
    want = [oracle.Dfa.from_spec(s).run(x) for s in gspecs]
    assert g.match(x) == want
    checked += 2 * len(gspecs)
    g.close()
    print("debug-bounds parity ok: %d checks" % checked)


if __name__ == "__main__":
    main()
