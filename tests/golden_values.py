"""Reader of the text fixtures under tests/golden/ (published values with their
citations in each file's header).  Lines starting with '#' are comments."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    """Whitespace-separated fields of every data line of tests/golden/<name>."""
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]


def values(name):
    """{first field: float(second field)} of a name/value fixture."""
    return {r[0]: float(r[1]) for r in rows(name)}


def philox_kat():
    """[(counter[4], key[2], output[4])] of the Philox4x32-10 known-answer fixture."""
    out = []
    for r in rows("philox4x32_10_kat.txt"):
        w = [int(x, 16) for x in r]
        out.append((w[0:4], w[4:6], w[6:10]))
    return out


def units():
    """Constants of the eV / A / fs / u / e / K unit system derived from the SI
    values: hbar (eV fs), k_B (eV/K), u A^2/fs^2 in eV, e^2/(4 pi eps0) in eV A."""
    import math
    si = values("codata2018_si.txt")
    e = si["e"]
    return {
        "hbar": si["h"] / (2 * math.pi) / e * 1e15,
        "k_B": si["k_B"] / e,
        "mvv2e": si["u"] * 1e-20 / 1e-30 / e,
        "k_e": e / (4 * math.pi * si["eps0"]) * 1e10,
    }
