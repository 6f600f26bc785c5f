"""Runs oracle jobs in a pool of spawned single-threaded processes (one per
host core), for GPU tests whose oracle side would otherwise take minutes.
Spawned, never forked: a process forked after the first GPU call can hang."""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")


def oracle_map(fn, jobs):
    """[fn(job) for job in jobs], in parallel; fn must be a module-level
    function of an importable module."""
    import multiprocessing as mp
    jobs = list(jobs)
    n = max(1, min(len(jobs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(fn, jobs, chunksize=1)


def energy_and_adjoint_of_weighted_score(job):
    """(sum w |W f|^2, Re W^*(2 w W f)) of one volume with the oracle:
    job = (f, w, dims, subdiv, L)."""
    from oracle import os3d_oracle as O
    f, w, dims, subdiv, L = job
    ob = O.Bank(dims, O.icosa_orientations(subdiv), O.Params(L=L))
    U = O.forward(f, ob)
    return O.weighted_energy(U, w), O.adjoint(O.weighted_energy_grad(U, w), ob)


def upsilon_of(job):
    """The oracle's Upsilon f = W^{*,ext} Phi W f: job = (f, dims, subdiv, L, power)."""
    from oracle import os3d_oracle as O
    f, dims, subdiv, L, power = job
    ob = O.Bank(dims, O.icosa_orientations(subdiv), O.Params(L=L))
    return O.upsilon(f, ob, power)
