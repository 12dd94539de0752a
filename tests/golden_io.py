"""Readers for the text fixtures under tests/golden/ (values typed from the paper)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln


def sections(name):
    """{section: [lines]} for files made of [name] headers."""
    out, cur = {}, None
    for ln in _lines(name):
        if ln.startswith("[") and ln.endswith("]"):
            cur = ln[1:-1]
            out[cur] = []
        else:
            out[cur].append(ln)
    return out


def matrix(lines):
    return np.array([[int(v) for v in ln.split()] for ln in lines], dtype=np.int64)


def table1():
    """{name: dict(T=int matrix, s=float vector, rho_lo, rho_hi)}"""
    out = {}
    for name, lines in sections("table1_rklt8.txt").items():
        d = {}
        rows = []
        for ln in lines:
            k, *rest = ln.split()
            if k in ("rho_lo", "rho_hi"):
                d[k] = float(rest[0])
            elif k == "s_recip_sq":
                d["s"] = 1.0 / np.sqrt(np.array([float(v) for v in rest]))
            else:
                rows.append(ln)
        d["T"] = matrix(rows)
        out[name] = d
    return out


def factors():
    return {k: matrix(v) for k, v in sections("fast_factorisation_n8.txt").items()}


def jpeg_zigzag():
    return np.array([[int(v) for v in ln.split()] for ln in _lines("jpeg_zigzag_8x8.txt")])


def table2():
    rows, rdct = [], None
    for ln in _lines("table2_measures.txt"):
        p = ln.split()
        if p[0] == "RDCT":
            rdct = dict(rho=float(p[1]), eps=float(p[2]), mse=float(p[3]))
        else:
            rows.append(dict(name=p[0], rho=float(p[1]), cg=float(p[2]), eta=float(p[3]),
                             eps=float(p[4]), mse=float(p[5])))
    return rows, rdct


def table3():
    return [dict(t=p[0], image=p[1], mse=float(p[2]), psnr=float(p[3]))
            for p in (ln.split() for ln in _lines("table3_mse_psnr.txt"))]
