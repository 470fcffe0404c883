"""The truth tables of the three-input logic instructions the stage rules
are written with (csrc/device_common.cuh): each named LUT constant equals
its documented formula evaluated on the operand patterns a = 0xF0,
b = 0xCC, c = 0xAA, so a wrong table fails here, before any GPU run."""
import os
import re

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1804_07981_b300", "csrc", "device_common.cuh")


def _tables():
    out = {}
    pat = re.compile(r"constexpr unsigned (k\w+) = (0x[0-9A-Fa-f]+);\s*//\s*(.*)$")
    with open(HDR) as f:
        for line in f:
            m = pat.search(line)
            if m:
                formula = m.group(3).replace("(c unused)", "").strip()
                out[m.group(1)] = (int(m.group(2), 16), formula)
    return out


def test_every_lut_matches_its_formula():
    tabs = _tables()
    assert {"kNor", "kNorAnd", "kAnd", "kAndNor", "kXor3", "kAndNotOr", "kAndOrNot",
            "kAndNand"} <= set(tabs)
    env = {"a": 0xF0, "b": 0xCC, "c": 0xAA}
    for name, (lut, formula) in tabs.items():
        assert re.fullmatch(r"[abc~&|^() ]+", formula), (name, formula)
        assert eval(formula, {}, env) & 0xFF == lut, (name, formula, hex(lut))


def test_the_rule_lines_in_lut_form_agree_with_plain_logic():
    """The Model I pair-stage lines, bit for bit on random words: the LUT
    forms used in the kernel against the plain expressions."""
    import random
    rng = random.Random(7)
    tabs = {k: v[0] for k, v in _tables().items()}
    M = 0xFFFFFFFF

    def lop3(lut, a, b, c):
        r = 0
        for i in range(32):
            idx = ((a >> i) & 1) << 2 | ((b >> i) & 1) << 1 | ((c >> i) & 1)
            r |= ((lut >> idx) & 1) << i
        return r

    for _ in range(200):
        L0, L2, T0, T2, sT, sM, X = (rng.getrandbits(32) for _ in range(7))
        assert lop3(tabs["kNor"], L0, T0, 0) == ~(L0 | T0) & M
        assert lop3(tabs["kAndNor"], L0, L2, T2) == L0 & ~(L2 | T2) & M
        assert lop3(tabs["kXor3"], L0, L2, X) == L0 ^ L2 ^ X
        assert lop3(tabs["kAndNotOr"], sT, X, sM) == ((sT & ~X) | sM) & M
        assert lop3(tabs["kNorAnd"], L0, T0, X) == ~(L0 | T0) & X & M
        assert lop3(tabs["kAndOrNot"], X, sT, sM) == X & (~sT | sM) & M
        assert lop3(tabs["kAndNand"], sT, X, sM) == sT & ~(X & sM) & M
        assert lop3(tabs["kAnd"], L0, X, 0) == L0 & X
