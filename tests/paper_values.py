"""Reader for the values the paper prints (tests/golden/)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table1():
    """Rows of Table 1 (Sec. 3.1) as dicts."""
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_table1.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        src, n, mid, s_cpu, s_gpu, p_high, p_all = line.split()
        rows.append(dict(source=src, histories=int(float(n)), middle=mid, sigma_cpu=float(s_cpu) / 100,
                         sigma_gpu=float(s_gpu) / 100, p_high=float(p_high) / 100,
                         p_all=float(p_all) / 100))
    return rows
