"""Host-side checks of the CUDA library (no GPU needed): the C ABI loads and
exports every entry point declared in include/nmpc.h, and the one-time
structure analysis (ordering, elimination tree, supernodes, level sets) is a
valid symbolic factorization of the condensed pattern, checked against the
oracle's SymCholesky (Sec. 3.2.3)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_2606_04725_gb300 as P
    P.build()
    return P


def test_library_exports_every_declared_symbol(P):
    header = open(os.path.join(ROOT, "include", "nmpc.h")).read()
    declared = set(re.findall(r"\b(nmpc_[a-z0-9_]+)\s*\(", header))
    lib = P.lib()
    missing = [name for name in sorted(declared) if not hasattr(lib, name)]
    assert not missing, missing
    assert declared == set(P._lib.EXPORTED)


def _header_struct_fields(header, name):
    """Field names, in order, of `typedef struct { ... } name;` in the header."""
    end = re.search(r"\}\s*" + name + r";", header).start()
    body = header[header.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    body = re.sub(r"\[[^]]*\]", "", body)  # array extents
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "double a, b, c" / "const int* horizons" / "struct {...} cand[16]"
        parts = decl.split(",")
        names.append(re.findall(r"\w+", parts[0])[-1])
        names.extend(re.findall(r"\w+", p)[-1] for p in parts[1:])
    return names


def test_binding_structs_mirror_the_header(P):
    """The ctypes structures lay out the header's structs field by field as
    it declares them."""
    header = open(os.path.join(ROOT, "include", "nmpc.h")).read()
    L = P._lib
    for cname, pyst in (("nmpc_problem", L.Problem), ("nmpc_options", L.Options),
                        ("nmpc_info", L.Info), ("nmpc_stats", L.Stats),
                        ("nmpc_tune_candidate", L.TuneCandidate), ("nmpc_tune_report", L.TuneReport),
                        ("nmpc_phase_times", L.PhaseTimes)):
        assert _header_struct_fields(header, cname) == [f[0] for f in pyst._fields_], cname


def test_problem_defaults_leave_the_control_tracking_cost_out(P):
    import ctypes as C
    p = P._lib.Problem()
    P.lib().nmpc_problem_defaults(0, C.byref(p))
    assert (p.wu, p.ubar, p.wdu, p.dt, p.N, p.Nf) == (0.0, 0.0, 0.01, 1.0, 12, 5)


CASES = [
    ("distill_nd", dict(model=0, horizons=[20], N=12, Nf=5), dict(ordering=2)),
    ("distill_nat", dict(model=0, horizons=[20], N=12, Nf=5), dict(ordering=1)),
    ("distill_batch", dict(model=0, horizons=[3, 7, 5], N=6, Nf=3), dict(ordering=0)),
    ("plate", dict(model=1, horizons=[4], g=8, S=8), dict(ordering=2)),
    ("toy", dict(model=2, horizons=[14]), dict(ordering=2)),
    ("distill_paper", dict(model=0, horizons=[90], N=32, Nf=17, dt=2.0, Ac=0.5, At=0.25, Ar=1.0, wdu=0.0,
                           wu=0.1, ubar=2.51459), dict(ordering=2)),
]


@pytest.mark.parametrize("name,prob,opt", CASES, ids=[c[0] for c in CASES])
def test_supernodal_structure_covers_symbolic_factor(P, oracle, name, prob, opt):
    s = P.Structure(opts=P.options(**opt), **prob)
    st = s.stats()
    n = st["n_total"]
    perm = s.export(0)
    assert sorted(perm.tolist()) == list(range(n))
    pairs = s.export(8)              # condensed pattern in factor order, lower
    assert np.all(pairs[:, 0] >= pairs[:, 1])
    assert len({(a, b) for a, b in pairs}) == len(pairs)
    assert np.all(np.isin(np.arange(n), pairs[pairs[:, 0] == pairs[:, 1], 0]))  # full diagonal
    # oracle symbolic factorization of the same pattern
    cols = [[] for _ in range(n)]
    for r, c in pairs:
        cols[c].append(r)
    colptr = np.cumsum([0] + [len(c) for c in cols])
    rowidx = np.concatenate([np.sort(c) for c in cols]).astype(np.int32)
    parent, Lp, Li = oracle.symbolic(n, colptr, rowidx)
    first, ncol, nrow = s.export(1), s.export(2), s.export(3)
    rows = s.export(4)
    sparent = s.export(5)
    rowptr = np.concatenate([[0], np.cumsum(nrow)])
    sn_of = np.empty(n, dtype=int)
    for k in range(len(first)):
        sn_of[first[k]:first[k] + ncol[k]] = k
        R = rows[rowptr[k]:rowptr[k + 1]]
        assert np.all(np.diff(R) > 0)
        np.testing.assert_array_equal(R[:ncol[k]], np.arange(first[k], first[k] + ncol[k]))
    assert np.all(np.diff(first) > 0) and first[0] == 0 and first[-1] + ncol[-1] == n
    # every structural nonzero of L lies in its supernode's row list
    for j in range(n):
        k = sn_of[j]
        R = set(rows[rowptr[k]:rowptr[k + 1]].tolist())
        missing = set(Li[Lp[j]:Lp[j + 1]].tolist()) - R
        assert not missing, (name, j, missing)
    # supernodal tree agrees with the elimination tree
    for k in range(len(first)):
        last = first[k] + ncol[k] - 1
        if parent[last] < 0:
            assert sparent[k] == -1
        else:
            assert sparent[k] == sn_of[parent[last]]
        for j in range(first[k], last):
            assert parent[j] == j + 1  # columns inside a supernode form a chain
    # levels: children strictly below parents
    lptr, lsn = s.export(6), s.export(7)
    level = np.empty(len(first), dtype=int)
    for l in range(len(lptr) - 1):
        level[lsn[lptr[l]:lptr[l + 1]]] = l
    for k in range(len(first)):
        if sparent[k] >= 0:
            assert level[sparent[k]] > level[k]
    assert st["factor_flops"] > 0 and s.workspace_bytes() > 0


def test_nested_dissection_reduces_depth(P):
    nd = P.Structure(model=0, horizons=[200], N=34, Nf=17, opts=P.options(ordering=2)).stats()
    nat = P.Structure(model=0, horizons=[200], N=34, Nf=17, opts=P.options(ordering=1)).stats()
    assert nd["n_levels"] <= 12 < nat["n_levels"]


def test_invalid_problems_are_rejected(P):
    with pytest.raises(P.NmpcError):
        P.Structure(model=0, horizons=[10], N=12, Nf=12)   # feed tray must be inside the column
    with pytest.raises(P.NmpcError):
        P.Structure(model=1, horizons=[3], g=10, S=12)     # g % (S/4) != 0
    with pytest.raises(P.NmpcError):
        P.Structure(model=0, horizons=[0], N=12, Nf=5)


@pytest.mark.parametrize("name,prob,opt", CASES, ids=[c[0] for c in CASES])
def test_levels_order_every_child_before_its_parent(P, name, prob, opt):
    """The level sets (supernodes by height) put every supernode at a strictly
    lower level than its parent.  The factorization runs level by level and the
    persistent solves claim fronts in level order, waiting only on children
    (forward) or the parent (backward); both rely on this order."""
    kw = {k: v for k, v in prob.items() if k not in ("model", "horizons")}
    s = P.Structure(prob["model"], prob["horizons"], opts=P.options(**opt), **kw)
    lp, ls, par = s.export(6), s.export(7), s.export(5)
    ns = len(par)
    assert sorted(ls.tolist()) == list(range(ns))
    level = np.empty(ns, dtype=int)
    for l in range(len(lp) - 1):
        level[ls[lp[l]:lp[l + 1]]] = l
    for j in range(ns):
        if par[j] >= 0:
            assert level[j] < level[par[j]], (j, par[j])
    # a front's rows are its columns followed by rows of its ancestors: the
    # update rows of a child are rows of its parent
    first, ncol, nrow = s.export(1), s.export(2), s.export(3)
    rows_ptr = np.concatenate([[0], np.cumsum(nrow)])
    rows = s.export(4)
    for j in range(ns):
        rj = rows[rows_ptr[j]:rows_ptr[j + 1]]
        assert np.array_equal(rj[:ncol[j]], np.arange(first[j], first[j] + ncol[j]))
        assert np.all(np.diff(rj) > 0)
        if par[j] >= 0:
            rp = set(rows[rows_ptr[par[j]]:rows_ptr[par[j] + 1]].tolist())
            assert set(rj[ncol[j]:].tolist()) <= rp, j


def test_batch_analysis_equals_each_instance_analysed_alone(P):
    """The batch analysis runs the symbolic work once per distinct horizon,
    on several host threads, and copies it to the other instances.  Every
    instance of an uneven batch with repeated horizons must then have the
    structure of the same horizon analysed alone: the same factor ordering
    (shifted by the instance's first variable), supernode sizes and row lists
    (shifted), and parents (shifted by its first supernode)."""
    hz = [50, 9, 80, 50, 9, 120, 80]
    kw = dict(N=12, Nf=5)
    b = P.Structure(P.MODEL_DISTILLATION, hz, **kw)
    perm_b, nc_b, nr_b = b.export(0), b.export(2), b.export(3)
    rows_b, par_b = b.export(4), b.export(5)
    vo = so = ro = 0
    for T in hz:
        s = P.Structure(P.MODEL_DISTILLATION, [T], **kw)
        perm, nc, nr, rows, par = s.export(0), s.export(2), s.export(3), s.export(4), s.export(5)
        n, ns, nrows = perm.size, nc.size, rows.size
        assert np.array_equal(perm_b[vo:vo + n], perm + vo)
        assert np.array_equal(nc_b[so:so + ns], nc) and np.array_equal(nr_b[so:so + ns], nr)
        assert np.array_equal(rows_b[ro:ro + nrows], rows + vo)
        assert np.array_equal(par_b[so:so + ns], np.where(par < 0, -1, par + so))
        vo, so, ro = vo + n, so + ns, ro + nrows
        s.close()
    assert vo == perm_b.size and so == nc_b.size


def test_automatic_amalgamation_keeps_small_separators_apart(P):
    """Automatic amalgamation: where every front of the relaxed partition is
    small (the distillation columns under nested dissection), the partition
    is the sibling-limited one, whose top separators are single stage blocks
    (x_k and u_k, N + 1 columns); where fronts are large (the heated plate at
    g = 32) it is the relaxed one.  Stage order gives a chain, where both
    modes agree.  Mode 2 only splits what mode 1 merged: every relaxed
    supernode is a union of sibling-limited ones."""
    def same(a, b):
        return all(np.array_equal(a.export(w), b.export(w)) for w in (0, 1, 2, 3, 5, 6, 7))

    auto, relaxed, sib = [P.Structure(model=0, horizons=[200], N=34, Nf=17, opts=P.options(ordering=2, amalgamation=am))
                          for am in (0, 1, 2)]
    assert same(auto, sib) and not same(relaxed, sib)
    assert max(relaxed.stats()["max_front"], sib.stats()["max_front"]) <= 128
    lp, lsn, ncol = sib.export(6), sib.export(7), sib.export(2)
    assert all(ncol[q] == 35 for q in lsn[lp[-4]:lp[-1]])       # the four top levels
    assert set(relaxed.export(1)) <= set(sib.export(1))           # relaxed = coarsening
    assert relaxed.stats()["nnz_L"] >= sib.stats()["nnz_L"]
    auto, relaxed, sib = [P.Structure(model=1, horizons=[20], g=32, S=8, opts=P.options(ordering=2, amalgamation=am))
                          for am in (0, 1, 2)]
    assert relaxed.stats()["max_front"] > 128 and same(auto, relaxed) and not same(relaxed, sib)
    chain = [P.Structure(model=0, horizons=[200], N=34, Nf=17, opts=P.options(ordering=1, amalgamation=am))
             for am in (0, 1, 2)]
    assert same(chain[0], chain[1]) and same(chain[1], chain[2])
    with pytest.raises(P.NmpcError):
        P.Structure(model=0, horizons=[20], N=12, Nf=5, opts=P.options(amalgamation=3))


def test_stats_report_the_amalgamation_used(P):
    used = [P.Structure(model=0, horizons=[200], N=34, Nf=17, opts=P.options(ordering=2, amalgamation=am))
            .stats()["amalgamation_used"] for am in (0, 1, 2)]
    assert used == [2, 1, 2]
    assert P.Structure(model=1, horizons=[20], g=32, S=8, opts=P.options(ordering=2)).stats()["amalgamation_used"] == 1


def test_library_and_oracle_default_to_the_same_model_constants(P, oracle):
    """Both sides solve the same problems by default: nmpc_problem_defaults
    and the oracle's problem constructors agree on every model constant and
    bound (the models of Sec. 4.1 with the benchmark readings)."""
    O = oracle
    fields = ("dt", "alpha", "D", "F", "xF", "Ac", "At", "Ar", "wdu", "wu", "ubar", "kappa", "cq", "rho_u",
              "xlo", "xhi", "ulo", "uhi")
    cases = [(0, O.distillation(12, 5, 3, np.zeros(12), np.zeros(3), 0.0)),
             (1, O.plate(8, 8, 2, np.zeros(64), np.zeros(64))),
             (2, O.toy(3, 1.0, np.zeros(3), dt=1.0))]
    for model, op in cases:
        gp, _ = P._lib.problem(model, [3])
        for f in fields:
            assert getattr(gp, f) == getattr(op._p, f), (model, f, getattr(gp, f), getattr(op._p, f))


@pytest.mark.parametrize("hz", [[200], [50 + 37 * (i % 5) for i in range(40)], [60 + (i * 7) % 140 for i in range(256)]])
def test_reduction_chunks_and_visiting_order(P, hz):
    """Reduction chunks partition every instance's variables and rows without
    crossing an instance, hold at most 128 E elements with E = clamp(total /
    (1216 x 128), 1, 16), and the reductions visit each variable chunk's
    variables longest Jacobian column first, ties in index order."""
    S = P.Structure(P.MODEL_DISTILLATION, hz, N=34, Nf=17)
    st = S.stats()
    n, m = st["n_total"], st["m_total"]
    E = max(1, min(16, (n + m) // (1216 * 128)))
    # instance offsets: x_0 plus (x_k, u_k) per stage; the initial rows plus N per stage
    voff = np.concatenate([[0], np.cumsum([34 + T * 35 for T in hz])])
    roff = np.concatenate([[0], np.cumsum([34 + T * 34 for T in hz])])
    assert voff[-1] == n and roff[-1] == m
    ch = S.export(9)
    order = S.export(10)
    clen = S.export(11)
    assert sorted(order.tolist()) == list(range(n))
    seen_v = np.zeros(n, dtype=int)
    seen_r = np.zeros(m, dtype=int)
    for inst, kind, b, e in ch:
        assert 0 < e - b <= 128 * E
        (seen_v if kind == 0 else seen_r)[b:e] += 1
        lo, hi = (voff[inst], voff[inst + 1]) if kind == 0 else (roff[inst], roff[inst + 1])
        assert lo <= b and e <= hi  # inside its own instance
        if kind == 0:
            vs = order[b:e]
            assert sorted(vs.tolist()) == list(range(b, e))  # the chunk's own variables
            key = [(-clen[v], v) for v in vs]
            assert key == sorted(key)
    assert (seen_v == 1).all() and (seen_r == 1).all()
    S.close()
