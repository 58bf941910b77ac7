"""Speed-up arithmetic of the paper's evaluation, used to report the GPU
analogue of its scaling study.

amdahl_speedup:        S_p = 1 / (r_s + r_p / p), r_p = 1 - r_s (Sec. II-B, Table I)
actual_speedup:        total time of one task / total time of N tasks (Eq. actualvst, Sec. V)
percentage_difference: |T - A| / ((T + A) / 2) * 100 (Eq. percen, Sec. V)
"""


def amdahl_speedup(r_s, p):
    """Theoretical speed-up on p tasks for serial fraction r_s (p = inf allowed)."""
    if p == float("inf"):
        return 1.0 / r_s
    return 1.0 / (r_s + (1.0 - r_s) / p)


def actual_speedup(t_single, t_multi):
    return t_single / t_multi


def percentage_difference(theoretical, actual):
    return abs(theoretical - actual) / ((theoretical + actual) / 2.0) * 100.0


def scaling_table(times, ideal=None):
    """times: {scheduler: {workers: seconds}} with workers = 1 present.
    Returns {scheduler: {workers: (speed-up, % difference vs ideal)}}; the
    ideal speed-up defaults to the worker count (r_s = 0)."""
    out = {}
    for sched, t in times.items():
        base = t[1]
        row = {}
        for w, tw in sorted(t.items()):
            a = actual_speedup(base, tw)
            th = ideal(w) if ideal else float(w)
            row[w] = (a, percentage_difference(th, a))
        out[sched] = row
    return out
