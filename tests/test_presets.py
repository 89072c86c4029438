"""The solver presets against the paper's printed settings (Sec. IV-D
parameters, Sec. IV-A iteration caps; tests/golden/paper_presets.txt), and
the library binding's presets against the oracle's."""
import dataclasses
import os

import oracle


def _paper_presets():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_presets.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows[f[0]] = dict(l=int(f[1]), t=int(f[2]), m=int(f[3]), rsd_limit=float(f[4]),
                              ndec_limit=int(f[5]), reldec_limit=float(f[6]), max_iter=int(f[7]),
                              restart=None if f[8] == "-" else int(f[8]), tol=float(f[9]))
    return rows


def test_paper_presets_are_the_printed_values():
    """PAPER_CG / PAPER_GMRES of the oracle and of the library binding carry the
    Sec. IV-D parameters and the Sec. IV-A iteration caps; the binding's four
    presets equal the oracle's field by field (the GPU parity tests run both
    sides under the same-named preset)."""
    from paper_2411_04686_gb300 import PAPER_CG, PAPER_GMRES, SCALED_CG, SCALED_GMRES
    ref = _paper_presets()
    for name, o, g in (("cg", oracle.PAPER_CG, PAPER_CG), ("gmres", oracle.PAPER_GMRES, PAPER_GMRES)):
        want = ref[name]
        for p in (o, g):
            for f in ("l", "t", "m", "rsd_limit", "ndec_limit", "reldec_limit", "max_iter"):
                assert getattr(p, f) == want[f], (name, f)
            if want["restart"] is not None:
                assert p.restart == want["restart"]
    for o, g in ((oracle.PAPER_CG, PAPER_CG), (oracle.PAPER_GMRES, PAPER_GMRES),
                 (oracle.SCALED_CG, SCALED_CG), (oracle.SCALED_GMRES, SCALED_GMRES)):
        assert dataclasses.asdict(o) == dataclasses.asdict(g)


def test_scaled_presets_keep_the_paper_thresholds():
    """The scaled presets (for systems that converge in hundreds of iterations)
    keep the paper's RSD and relDec limits and scale nDec_limit with t: the
    paper's nDec_limit / t ratio (130/250, 80/300) times the scaled t, rounded."""
    ref = _paper_presets()
    for name, p in (("cg", oracle.SCALED_CG), ("gmres", oracle.SCALED_GMRES)):
        want = ref[name]
        assert p.rsd_limit == want["rsd_limit"] and p.reldec_limit == want["reldec_limit"]
        assert p.ndec_limit == round(want["ndec_limit"] / want["t"] * p.t)
        assert p.l < want["l"] and p.t < want["t"] and p.m < want["m"]
