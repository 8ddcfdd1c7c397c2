"""Readers of the paper's printed values (the text fixtures beside this file)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE2_COLUMNS = ("hs", "cgcg", "m", "pr", "gv", "pipe_m", "pipe_pr")


def _rows(name):
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                yield line


def table1():
    """{variant: {vec, vec_pc, scal, products, mem, mem_pc}} (Table 1)."""
    keys = ("vec", "vec_pc", "scal", "products", "mem", "mem_pc")
    return {r[0]: dict(zip(keys, map(int, r[1:]))) for r in _rows("table1_costs.txt")}


def table2():
    """{"none" | "jacobi": {variant: (iterations to 1e5, min log10 error)}}
    (Table 2, row model_48_8_3)."""
    out = {}
    for r in _rows("table2_model_48_8_3.txt"):
        its, errs = r[1:8], r[8:15]
        out[r[0]] = {v: (int(i), float(e)) for v, i, e in zip(TABLE2_COLUMNS, its, errs)}
    return out
