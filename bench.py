#!/usr/bin/env python3
"""Throughput of the invertible 3D orientation-score transform on GB300.

One step = forward transform U = W f plus exact inverse f_rec = W^-1 U of one
synthetic 128^3 volume (12 spline tubes + noise) with N_o = 162 icosahedral
orientations, L = 16 (complex64 scores, 2.72 GB, larger than L2).
Metric: voxel-orientations per second = n^3 N_o / (t_fwd + t_inv).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): independent replicas, one volume per
rank per step, no collective on the data path ("scaling": "weak").
The reference arm (--impl reference) times the FP64 CPU oracle on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the oracle runs as one single-threaded process per host core: keep numpy's
# BLAS to one thread in each (the spawned workers inherit this)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

WORKLOAD = "splines128_no162"
METRIC = "OS transform voxel·orientations/s (fwd+inv, FP32) at 128³×162; p50/p99 latency"
UNIT = "voxel-orientations/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bf16", action="store_true", help="store U as bfloat16 pairs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--block-slots", type=int, default=0,
                    help="orientation pairs per launch block (0 = the library's choice)")
    ap.add_argument("--serve", type=int, default=0,
                    help="instead of the headline: serve this many Poisson-arriving requests "
                         "of the mixed-size workload and report p50/p99 latency")
    ap.add_argument("--load", type=float, default=0.8,
                    help="--serve arrival rate as a fraction of the measured capacity")
    ap.add_argument("--precision", action="store_true",
                    help="instead of the headline: reconstruction error of complex64 and BF16 "
                         "scores at 256^3 x 42 against the exact result")
    ap.add_argument("--only-step", action="store_true",
                    help="time the headline step alone (no end-to-end, per-kernel, operation, "
                         "serving, precision or CPU legs): for profiler captures")
    ap.add_argument("--only-op", default="", choices=["", "enhance_linear_162", "enhance_linear_42", "upsilon",
                                                  "autograd", "score_energy"],
                    help="time one operation alone on the headline grid (for profiler captures): "
                         "enhance_linear_162 = the linear diffusion with the 162-orientation bank; "
                         "upsilon = the fused soft-threshold processing (p = 1.5)")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="named synthetic workload (default: the 128^3 x 162 headline)")
    return ap.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _workload_setup():
    from paper_1505_07690_gb300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    return w, synth


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, pci_bus_id):
        self.pci = pci_bus_id
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "50"]
            if self.pci:
                cmd += ["-i", self.pci]
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = list(csv.reader(io.StringIO(self.tmp.read())))
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on all host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
_OW = {}


def _ow_init(dims, orients, L, shm_in, shm_out, slots):
    import numpy as np
    from multiprocessing import shared_memory
    from oracle import os3d_oracle as O
    _OW["O"] = O
    _OW["bank"] = O.Bank(dims, orients, O.Params(L=L))
    _OW["shm"] = (shared_memory.SharedMemory(name=shm_in), shared_memory.SharedMemory(name=shm_out))
    _OW["f"] = np.ndarray(dims, np.float64, buffer=_OW["shm"][0].buf)
    _OW["out"] = np.ndarray((slots,) + tuple(dims), np.complex128, buffer=_OW["shm"][1].buf)


def _ow_m_part(job):
    slot, idx = job
    _OW["out"][slot] = _OW["bank"].M_part(idx)
    return slot


def _ow_transform_part(job):
    """The oracle's forward transform of the shared volume for the
    orientations idx, then their part of the inverse's orientation sum."""
    slot, idx = job
    O, bank = _OW["O"], _OW["bank"]
    U = O.forward(_OW["f"], bank, idx)
    _OW["out"][slot] = O.backproject(U, bank, idx)
    return slot


def _ow_init_in(dims, orients, L, shm_in):
    import numpy as np
    from multiprocessing import shared_memory
    from oracle import os3d_oracle as O
    _OW["O"] = O
    _OW["bank"] = O.Bank(dims, orients, O.Params(L=L))
    _OW["shm"] = (shared_memory.SharedMemory(name=shm_in),)
    _OW["f"] = np.ndarray(dims, np.float64, buffer=_OW["shm"][0].buf)


def _ow_sample_part(i):
    """The oracle's forward transform of the shared volume for orientation i
    and that orientation's part of the inverse's orientation sum; (seconds,
    checksum)."""
    import numpy as np
    O, bank = _OW["O"], _OW["bank"]
    t0 = time.perf_counter()
    U = O.forward(_OW["f"], bank, [i])
    acc = O.backproject(U, bank, [i])
    return time.perf_counter() - t0, float(np.abs(acc).sum())


def oracle_sample_on_cores(workload, cores=None):
    """The oracle on a bounded sample of a large workload: one orientation per
    single-threaded process (as many as host cores and memory allow, about
    2 GB each at 256^3), each the forward transform of the whole volume and
    its part of the inverse's orientation sum. (voxel-orientations/s over the
    slowest process's time, description, processes)."""
    import multiprocessing as mp
    import numpy as np
    from multiprocessing import shared_memory
    from oracle import os3d_oracle as O
    from paper_1505_07690_gb300 import synth
    w = synth.WORKLOADS[workload]
    dims = tuple(w["shape"])
    nvox = int(np.prod(dims))
    V = O.icosa_orientations(w["subdiv"])
    try:
        ram = os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        ram = 0
    per_proc = 16 * nvox * 8          # the volume and its transforms in complex128
    n = max(1, min(cores or os.cpu_count() or 1, len(V), int(0.3 * ram // per_proc) or 1))
    f = synth.workload_volume(workload).astype(np.float64)
    shm = shared_memory.SharedMemory(create=True, size=nvox * 8)
    try:
        np.ndarray(dims, np.float64, buffer=shm.buf)[...] = f
        with mp.get_context("spawn").Pool(n, initializer=_ow_init_in,
                                          initargs=(dims, V, w["L"], shm.name)) as pool:
            res = pool.map(_ow_sample_part, list(range(n)), chunksize=1)
    finally:
        shm.close()
        shm.unlink()
    t = max(r[0] for r in res)
    grid = "x".join(str(d) for d in dims)
    desc = (f"{n} of the {len(V)} orientations of the whole {grid} volume ({workload}): per "
            f"orientation the forward transform and its part of the exact inverse's orientation "
            f"sum (the inverse's last per-volume step, 1/{len(V)} of its work, left out), one "
            f"orientation per single-threaded numpy FP64 process, slowest {t:.1f} s")
    return n * nvox / t, desc, n


class OracleOnCores:
    """The FP64 oracle's forward transform and exact inverse of one volume,
    its orientations dealt over one single-threaded process per host core
    (spawned, so that no process is forked after the first GPU call). The
    orientation sums of the inverse and of M are added up from the parts and
    the last step of the inverse runs here: the result is the oracle's
    inverse(forward(f)) up to the order of the orientation sum."""

    def __init__(self, dims, orients, L, f, cores=None):
        import multiprocessing as mp
        import numpy as np
        from multiprocessing import shared_memory
        from oracle import os3d_oracle as O
        self.O = O
        self.dims = tuple(int(d) for d in dims)
        orients = np.asarray(orients, dtype=np.float64)
        n_o = len(orients)
        self.cores = max(1, min(cores or os.cpu_count() or 1, n_o))
        self.parts = [list(range(k, n_o, self.cores)) for k in range(self.cores)]
        nvox = int(np.prod(self.dims))
        self.shm_in = shared_memory.SharedMemory(create=True, size=nvox * 8)
        self.shm_out = shared_memory.SharedMemory(create=True, size=self.cores * nvox * 16)
        self.f = np.ndarray(self.dims, np.float64, buffer=self.shm_in.buf)
        self.f[...] = f
        self.out = np.ndarray((self.cores,) + self.dims, np.complex128, buffer=self.shm_out.buf)
        self.bank = O.Bank(self.dims, orients, O.Params(L=L))
        self.pool = mp.get_context("spawn").Pool(
            self.cores, initializer=_ow_init,
            initargs=(self.dims, orients, L, self.shm_in.name, self.shm_out.name, self.cores))
        # bank construction (untimed, as on the GPU): M from its parts
        self.pool.map(_ow_m_part, list(enumerate(self.parts)), chunksize=1)
        self.bank.set_M(self.out.real.sum(axis=0))

    def step(self):
        """One forward + exact inverse; (f_rec, seconds)."""
        t0 = time.perf_counter()
        self.pool.map(_ow_transform_part, list(enumerate(self.parts)), chunksize=1)
        f_rec = self.O.reconstruct(self.out.sum(axis=0), self.bank)
        return f_rec, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()
        del self.f, self.out
        for m in (self.shm_in, self.shm_out):
            m.close()
            m.unlink()


def oracle_on_cores(workload, steps=1, cores=None):
    """(voxel-orientations/s, f_rec, description) of the oracle on the whole
    named workload (all its orientations, forward + inverse) on the host cores."""
    import numpy as np
    from oracle import os3d_oracle as O
    from paper_1505_07690_gb300 import synth
    w = synth.WORKLOADS[workload]
    f = synth.workload_volume(workload).astype(np.float64)
    V = O.icosa_orientations(w["subdiv"])
    oc = OracleOnCores(w["shape"], V, w["L"], f, cores)
    try:
        dt = 0.0
        for _ in range(steps):
            f_rec, t = oc.step()
            dt += t
    finally:
        oc.close()
    nvox = int(np.prod(w["shape"]))
    grid = "x".join(str(n) for n in w["shape"])
    desc = (f"the whole {grid} x {len(V)} workload ({workload}), forward + exact inverse, "
            f"{steps} step(s) in {dt:.1f} s; orientations split over {oc.cores} single-threaded "
            f"numpy FP64 processes")
    return nvox * len(V) * steps / dt, f_rec, desc, oc.cores


def _config(dims, n_o, L, udtype="c64", world=1):
    nvox = int(dims[0] * dims[1] * dims[2])
    esize = 4 if udtype == "bf16x2" else 8
    return {"workload": WORKLOAD, "dims": list(dims), "n_o": n_o, "L": L, "batch_per_gpu": 1,
            "udtype": udtype, "parallelism": f"replicas{world}",
            "l2": f"inputs larger than L2 (U = {n_o * nvox * esize / 1e9:.2f} GB)"}


def run_reference(args):
    """The oracle as the reference arm: every step is the whole workload
    (forward + exact inverse of one volume with all its orientations) on all
    host cores; rank 0 only."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import os3d_oracle as O
    from paper_1505_07690_gb300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    f = synth.workload_volume(WORKLOAD).astype(np.float64)
    V = O.icosa_orientations(w["subdiv"])
    oc = OracleOnCores(w["shape"], V, w["L"], f)
    try:
        for _ in range(args.warmup):
            oc.step()
        times = [oc.step()[1] for _ in range(args.steps)]
    finally:
        oc.close()
    tot = sum(times)
    nvox = int(np.prod(w["shape"]))
    value = nvox * len(V) * args.steps / tot
    desc = (f"every step the whole workload: forward + exact inverse of one volume with all "
            f"{len(V)} orientations, split over {oc.cores} single-threaded numpy FP64 processes")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(w["shape"], len(V), w["L"], world=world),
        "latency_ms": {"p50": 1e3 * float(np.percentile(times, 50)),
                       "p99": 1e3 * float(np.percentile(times, 99))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oc.cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
def _code_lines(text):
    """Source text without // comments, trailing blanks and empty lines (the
    kernel sources hold no // inside string literals)."""
    out = []
    for line in text.splitlines():
        line = line.split("//", 1)[0].rstrip()
        if line:
            out.append(line)
    return "\n".join(out)


def _source_hash():
    """sha256[:12] of the kernel sources (file names and code, comments
    excluded): a recorded ncu figure stays valid while this is unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1505_07690_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if not f.endswith((".cu", ".cuh", ".h")):
            continue
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(f.encode() + b"\0" + _code_lines(fh.read()).encode() + b"\0")
    return h.hexdigest()[:12]


def _ncu_traffic(kind):
    """DRAM bytes per launch of ``kind`` from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    src = _source_hash()
    for line in open(path):
        p = line.split()
        if len(p) >= 4 and not line.startswith("#") and p[0] == kind and p[1] == WORKLOAD:
            return float(p[3]) if p[2] == src else None
    return None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _max_over_ranks(value, device):
    """The maximum of ``value`` over the ranks of the default process group
    (the value itself when there is none)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _cufft_compare(os3d, bank, V, dims, w, f, frec, steps, timed):
    """Forward + exact inverse with torch.fft (cuFFT, batched over the N_o
    orientations) and elementwise products with stored wavelets; the timing
    and the relative L2 difference of its reconstruction from ours."""
    import math
    import torch
    dev = f.device
    _, c = os3d.os3d_bank_coefficients(bank)
    minv = os3d.os3d_bank_minv(bank)
    k = [torch.fft.fftfreq(n, device=dev, dtype=torch.float64) * 2 * math.pi for n in dims]
    wz, wy, wx = k[0][:, None, None], k[1][None, :, None], k[2][None, None, :]
    r2 = wz ** 2 + wy ** 2 + wx ** 2
    N, gamma = bank.params.N, bank.params.gamma
    x = r2 / (2 * (gamma * math.pi) ** 2 / (1 + 2 * N))
    g = torch.zeros_like(x)
    term = torch.ones_like(x)
    for q in range(N + 1):
        if q:
            term = term * x / q
        g = g + term
    G = torch.where(r2 < math.pi ** 2, torch.exp(-x) * g, torch.zeros_like(x))
    ri = torch.where(r2 > 0, torch.rsqrt(torch.where(r2 > 0, r2, torch.ones_like(r2))),
                     torch.zeros_like(r2))
    psi = torch.empty((len(V),) + tuple(dims), device=dev, dtype=torch.float32)
    for i, (nx, ny, nz) in enumerate(V):
        t = ((wx * nx + wy * ny + wz * nz) * ri).clamp(-1, 1)
        pm, pl = torch.ones_like(t), t
        h = c[0] * pm + (c[1] * pl if len(c) > 1 else 0)
        for l in range(1, len(c) - 1):
            pm, pl = pl, ((2 * l + 1) * t * pl - l * pm) / (l + 1)
            h = h + c[l + 1] * pl
        h = torch.where(r2 > 0, h, torch.full_like(h, c[0]))
        psi[i] = (G * h).float()
    del wz, wy, wx, r2, x, g, term, ri
    fin = f[0]
    out = torch.empty_like(fin)

    def step():
        fh = torch.fft.fftn(fin)
        U = torch.fft.ifftn(fh[None] * psi, dim=(-3, -2, -1))
        A = (torch.fft.fftn(U, dim=(-3, -2, -1)) * psi).sum(0)
        out.copy_(torch.fft.ifftn(A * minv).real)

    # best of three rounds: its multi-GB temporaries go through torch's
    # caching allocator, whose state varies from round to round
    ms = min(timed(step, max(2, steps // 2)) for _ in range(3))
    ref = frec[0]
    diff = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
    # the same with the antipodal pairing (orientation i + N_o/2 = -n_i): one
    # transform per pair each way, U_b = conj U_a written out as well
    h = len(V) // 2
    Ufull = torch.empty((len(V),) + tuple(dims), device=dev, dtype=torch.complex64)
    out2 = torch.empty_like(fin)

    def step_paired():
        fh = torch.fft.fftn(fin)
        Ua = torch.fft.ifftn(fh[None] * psi[:h], dim=(-3, -2, -1))
        Ufull[:h] = Ua
        Ufull[h:] = Ua.conj()
        A = (torch.fft.fftn(Ufull[:h] + Ufull[h:].conj(), dim=(-3, -2, -1)) * psi[:h]).sum(0)
        out2.copy_(torch.fft.ifftn(A * minv).real)

    ms2 = min(timed(step_paired, max(2, steps // 2)) for _ in range(3))
    diff2 = float(torch.linalg.vector_norm(out2 - ref) / torch.linalg.vector_norm(ref))
    nvox = int(math.prod(dims))
    del psi, Ufull
    torch.cuda.empty_cache()
    return {"ms": ms, "value": nvox * len(V) / (ms / 1e3), "unit": UNIT,
            "library": "cuFFT via torch.fft (comparison only)",
            "recon_rel_l2_vs_ours": diff,
            "paired_ms": ms2, "paired_value": nvox * len(V) / (ms2 / 1e3),
            "paired_recon_rel_l2_vs_ours": diff2}


def _autograd_step(os3d, synth, steps, timed):
    """One loss.backward() of L = sum w |W f|^2 for a batch of 8 96^3 volumes
    with 42 orientations: os3d_forward plus os3d_adjoint behind
    torch.autograd."""
    import numpy as np
    import torch
    from paper_1505_07690_gb300.autograd import orientation_score, score_energy, weighted_energy
    w = synth.WORKLOADS["splines96x8_no42"]
    dims, B = w["shape"], w["batch"]
    V = os3d.os3d_icosa_orientations(w["subdiv"])
    bank = os3d.os3d_make_wavelets(dims, V, os3d.os3d_default_params(L=w["L"]))
    f = torch.from_numpy(np.stack([synth.workload_volume("splines96x8_no42", batch_index=b)
                                   for b in range(B)])).cuda().requires_grad_(True)
    wt = torch.from_numpy(synth.score_weights((B, len(V)) + tuple(dims), seed=1)).cuda()

    def step_torch_loss():
        f.grad = None
        U = orientation_score(f, bank)
        (wt * (U.real ** 2 + U.imag ** 2)).sum().backward()

    def step_energy():
        f.grad = None
        weighted_energy(orientation_score(f, bank), wt).backward()

    def step_stored():
        f.grad = None
        score_energy(f, bank, wt, sweep=False).backward()

    def step():
        f.grad = None
        score_energy(f, bank, wt).backward()

    ms_torch = timed(step_torch_loss, max(2, steps // 2))
    ms_energy = timed(step_energy, max(2, steps // 2))
    ms_stored = timed(step_stored, max(2, steps // 2))
    os3d.os3d_profile_reset()
    os3d.os3d_profile_enable(True)
    ms = timed(step, max(2, steps // 2))
    torch.cuda.synchronize()
    os3d.os3d_profile_enable(False)
    prof = os3d.os3d_profile_read()
    fd = f.detach()
    U = os3d.new_score(bank, B)
    g = torch.empty_like(fd)

    def transforms():
        os3d.os3d_forward(bank, fd, U)
        os3d.os3d_adjoint(bank, U, g)

    ms_t = timed(transforms, max(2, steps // 2))
    vo = B * int(np.prod(dims)) * len(V)
    del f, wt, U, g, fd
    torch.cuda.empty_cache()
    kinds = {k: v for k, v in prof.items() if v[0] > 0}
    calls = max(prof["weighted_energy"][0], 1)   # one final energy sum per step
    return {"ms": ms, "value": vo / (ms / 1e3), "unit": UNIT,
            "what": "score_energy: one sweep per block (forward z-pass, plane pass forming U "
                    "in shared memory, summing w|U|^2 and weighting it by 2w, adjoint "
                    "z-pass), no stored score; backward scales the gradient by g; batch 8",
            "kernels_per_step": {k: {"launches": v[0] / calls, "ms": v[1] / calls}
                                 for k, v in kinds.items()},
            "stored_score_ms": ms_stored,
            "stored_score_what": "score_energy(sweep=False): os3d_forward, weighted energy "
                                 "kernel, weighted adjoint (2 g w U folded into the plane pass)",
            "energy_then_adjoint_ms": ms_energy,
            "energy_then_adjoint_what": "orientation_score + weighted_energy: the gradient "
                                        "2 g w U stored, then os3d_adjoint",
            "torch_loss_ms": ms_torch, "torch_loss_value": vo / (ms_torch / 1e3),
            "transforms_ms": ms_t, "transforms_value": vo / (ms_t / 1e3)}


# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1505_07690_gb300 import build, os3d
    if rank == 0 or not os.path.exists(os3d.LIB_PATH):
        build.build()
    if world > 1:
        torch.distributed.barrier()

    w, synth = _workload_setup()
    dims = w["shape"]
    f_np = synth.workload_volume(WORKLOAD, seed=0, batch_index=rank)
    V = os3d.os3d_icosa_orientations(w["subdiv"])
    n_o = len(V)
    bank = os3d.os3d_make_wavelets(dims, V, os3d.os3d_default_params(L=w["L"],
                                                                      block_slots=args.block_slots))
    f = torch.from_numpy(f_np).cuda().unsqueeze(0)
    U = os3d.new_score(bank, 1, bf16=args.bf16)
    frec = torch.empty_like(f)
    stream = torch.cuda.current_stream()
    nvox = int(np.prod(dims))
    esize = 4 if args.bf16 else 8

    def step():
        os3d.os3d_forward(bank, f, U)
        os3d.os3d_inverse(bank, U, frec)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- timed region: K steps, device-side events, inputs resident in HBM
    clocks = ClockSampler(torch.cuda.get_device_properties(local).pci_bus_id
                          if hasattr(torch.cuda.get_device_properties(local), "pci_bus_id") else None)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    clocks.start()
    l0 = os3d.os3d_launch_count()
    ev[0].record(stream)
    for i in range(args.steps):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    launches = os3d.os3d_launch_count() - l0
    barrier()
    clk = clocks.stop()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = _max_over_ranks(ev[0].elapsed_time(ev[-1]), "cuda")
    value = world * nvox * n_o * args.steps / (total_ms / 1e3)
    if args.only_step:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": total_ms / args.steps, "only_step": True,
                              "config": _config(dims, n_o, w["L"], "bf16x2" if args.bf16 else "c64",
                                                world),
                              "gpu_launches": launches, "clocks": clk}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # ---- end to end: host buffers through the public API, copies timed.
    # Every step copies its input host -> device and its result device -> host
    # inside the timed region; the copies run on a second stream with two
    # device input buffers, so the upload for step i+1 overlaps step i.
    f_host = torch.from_numpy(f_np).unsqueeze(0).pin_memory()
    out_host = [torch.empty_like(f_host).pin_memory() for _ in range(2)]
    f_dev = [torch.empty_like(f) for _ in range(2)]
    frec2 = [torch.empty_like(f) for _ in range(2)]
    copy = torch.cuda.Stream()
    up = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]

    def upload(i):
        b = i % 2
        copy.wait_event(done[b])          # the buffer's previous step has read it
        with torch.cuda.stream(copy):
            f_dev[b].copy_(f_host, non_blocking=True)
            up[b].record(copy)

    def e2e_run(n):
        for b in range(2):
            done[b].record(stream)
        upload(0)
        for i in range(n):
            b = i % 2
            if i + 1 < n:
                upload(i + 1)
            stream.wait_event(up[b])
            os3d.os3d_forward(bank, f_dev[b], U)
            os3d.os3d_inverse(bank, U, frec2[b])
            done[b].record(stream)
            out_host[b].copy_(frec2[b], non_blocking=True)

    e2e_run(2)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(e0.elapsed_time(e1), "cuda")
    e2e_value = world * nvox * n_o * args.steps / (e2e_ms / 1e3)

    # ---- per-kernel durations (CUDA events around every launch, same stream)
    os3d.os3d_profile_reset()
    os3d.os3d_profile_enable(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    os3d.os3d_profile_enable(False)
    prof = os3d.os3d_profile_read()
    algo = {  # algorithmic HBM bytes over K steps, per kernel kind
        "xy_fwd_score": args.steps * n_o * nvox * esize,
        "xy_inv_score": args.steps * n_o * nvox * esize,
        "xy_fwd_real": args.steps * nvox * 4,
        "xy_inv_real": args.steps * nvox * 4,
    }
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    peaks, peak_kind = _peaks()
    nl, ms = prof[dom]
    if dom in algo and ms > 0:
        achieved = algo[dom] / (ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": _ncu_traffic(dom), "peak_source": peak_kind,
                "bytes_per_launch": algo[dom] / max(nl, 1), "launch_ms": ms / max(nl, 1)}
    else:
        roof = {"bound": "alu", "kernel": dom, "achieved": None, "peak": None, "unit": "TFLOP/s",
                "frac": None, "traffic": _ncu_traffic(dom), "launch_ms": ms / max(nl, 1)}
    # whole-step HBM view: U written once and read once
    step_bytes = 2 * n_o * nvox * esize + 4 * nvox * 4
    # algorithmic FP32 flops per step: per orientation pair (antipodal
    # pairing: one 3D transform per pair) and direction, a 3D DFT at
    # 5 n^3 log2(n^3) (radix-2 convention) plus the wavelet at every point,
    # 2 (L + 1) + 15 (Horner on L + 1 coefficients, the direction cosine, the
    # radial factor and the product)
    pairs = (n_o + 1) // 2
    step_flops = 2.0 * pairs * nvox * (5.0 * math.log2(nvox) + 2 * (w["L"] + 1) + 15)
    kernels = {k: {"launches": v[0], "ms_per_step": v[1] / args.steps,
                   "share": v[1] / max(sum(x[1] for x in prof.values()), 1e-9)}
               for k, v in prof.items() if v[0]}

    # ---- the score-domain operations on the same workload (CUDA events)
    def timed(fn, n):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    hbm = peaks["hbm_gbs"]
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    ops = {}
    ms_a = timed(lambda: os3d.os3d_approx_reconstruct(bank, U, frec), args.steps)
    by_a = n_o * nvox * esize + nvox * 4
    ops["approx_reconstruct"] = {"ms": ms_a, "bytes": by_a, "achieved_gbs": by_a / ms_a / 1e6,
                                 "frac_hbm": by_a / ms_a / 1e6 / hbm}
    ms_p = timed(lambda: os3d.os3d_project(bank, U, U), args.steps)
    ops["project"] = {"ms": ms_p, "value": nvox * n_o / (ms_p / 1e3), "unit": UNIT}
    ms_s = timed(lambda: os3d.os3d_soft_threshold(U, 1.5, out=U), args.steps)
    by_s = 2 * n_o * nvox * esize
    ops["soft_threshold"] = {"ms": ms_s, "bytes": by_s, "achieved_gbs": by_s / ms_s / 1e6,
                             "frac_hbm": by_s / ms_s / 1e6 / hbm}
    fu = torch.empty_like(f)
    ms_u = timed(lambda: os3d.os3d_upsilon(bank, f, 1.5, fu), args.steps)
    ops["upsilon_fused"] = {"ms": ms_u, "value": nvox * n_o / (ms_u / 1e3), "unit": UNIT,
                            "score_bytes_stored": 0}
    # cuFFT comparison (not the product path): the straightforward batched form,
    # f_hat = FFT(f), U = IFFT(f_hat psi_hat_i) for all i, then FFT of every U_i,
    # multiply, orientation sum, x M^-1, IFFT; psi_hat_i stored (setup untimed)
    os3d.os3d_forward(bank, f, U)          # our reconstruction, for the comparison's check
    os3d.os3d_inverse(bank, U, frec)
    ops["cufft_compare"] = _cufft_compare(os3d, bank, V, dims, w, f, frec, args.steps, timed)

    # differentiation form: 8 x 96^3, 42 orientations, loss sum w |U|^2 through
    # the autograd wrapper (forward, then the hand-written adjoint as backward)
    ops["autograd_8x96_no42"] = _autograd_step(os3d, synth, args.steps, timed)

    # linear diffusion: 42 orientations (the flows of Sec. 4.1 use N_o = 42), same grid
    V42 = os3d.os3d_icosa_orientations(1)
    bank42 = os3d.os3d_make_wavelets(dims, V42, os3d.os3d_default_params(L=w["L"]))
    dif = os3d.os3d_default_diffusion()
    os3d.os3d_profile_reset()
    os3d.os3d_profile_enable(True)
    ms_e = timed(lambda: os3d.os3d_enhance_linear(bank42, f, dif, fu), args.steps)
    torch.cuda.synchronize()
    os3d.os3d_profile_enable(False)
    pe = os3d.os3d_profile_read()["enhance_linear"]
    # algorithmic FP32 flops per in-ball frequency: K steps of an N_o x N_o
    # matrix-vector product (2 N_o^2) plus 2 N_o wavelet evaluations (Horner,
    # 2 x 17 flops each) and the spatial factors
    wz = np.fft.fftfreq(dims[0])[:, None, None] * 2 * np.pi
    wy = np.fft.fftfreq(dims[1])[None, :, None] * 2 * np.pi
    wx = np.fft.fftfreq(dims[2])[None, None, :] * 2 * np.pi
    inball = int(np.count_nonzero(wz ** 2 + wy ** 2 + wx ** 2 < np.pi ** 2))
    no42 = len(V42)
    # the kernel integrates half of the ball (the factor is even in w for an
    # antipodally closed set); counted with the real orientation count (the
    # kernel pads it to a multiple of 8 and executes more)
    flops = (inball + 1) // 2 * (dif.steps * 2 * no42 * no42 + 2 * no42 * 34 + no42 * 12)
    # executed: the kernel integrates the closed set as its 21 pairs, two
    # blocks of 24 rows (padded) over 22 columns each, and evaluates the even
    # or odd part of h once per row (17 flops per pair)
    pb, npair = 24, no42 // 2
    rows, cols = 2 * pb, (npair + 1) & ~1
    flops_exec = (inball + 1) // 2 * (dif.steps * 2 * rows * cols + 2 * npair * 34 + no42 * 12)
    k_ms = pe[1] / max(pe[0], 1)
    fp32_peak = nsm * 128 * 2 * (clk["sm_mhz"] if clk else 2070.0) * 1e6 / 1e12
    ops["enhance_linear"] = {
        "ms": ms_e, "n_o": no42, "steps": dif.steps,
        "value": nvox * no42 / (ms_e / 1e3), "unit": UNIT,
        "kernel_ms": k_ms, "bound": "alu", "kernel_tflops": flops / (k_ms / 1e3) / 1e12,
        "fp32_peak_tflops": fp32_peak,
        "frac_fp32": flops / (k_ms / 1e3) / 1e12 / fp32_peak,
        "executed_tflops": flops_exec / (k_ms / 1e3) / 1e12,
        "frac_fp32_executed": flops_exec / (k_ms / 1e3) / 1e12 / fp32_peak,
        "flops_note": "kernel_tflops counts the definition (the N_o x N_o propagator product, "
                      "2 N_o^2 per frequency and step); executed_tflops the pair-split "
                      "product the kernel runs (two blocks of N_o / 2)"}
    del bank42
    # the same flow for the 162-orientation headline bank: the propagator
    # product on the tensor cores (128 frequencies per MMA tile, 162 padded to
    # 176, three half-precision products per step for FP32 accuracy)
    os3d.os3d_profile_reset()
    os3d.os3d_profile_enable(True)
    ms_e2 = timed(lambda: os3d.os3d_enhance_linear(bank, f, dif, fu), args.steps)
    torch.cuda.synchronize()
    os3d.os3d_profile_enable(False)
    pe2 = os3d.os3d_profile_read()["enhance_linear"]
    k2 = pe2[1] / max(pe2[0], 1)
    half_ball = (inball + 1) // 2
    np_pad = 176
    tiles = (half_ball + 127) // 128
    mma_flops = tiles * dif.steps * 3 * 2 * 128 * np_pad * np_pad
    algo162 = half_ball * (dif.steps * 2 * n_o * n_o)
    ops["enhance_linear_162"] = {
        "ms": ms_e2, "n_o": n_o, "steps": dif.steps, "kernel_ms": k2,
        "value": nvox * n_o / (ms_e2 / 1e3), "unit": UNIT,
        "bound": "tensor", "tensor_tflops": mma_flops / (k2 / 1e3) / 1e12,
        "peak_tflops": peaks.get("bf16_tflops"), "peak_kind": "measured dense bf16 (f16 runs at the same rate), burst",
        "frac_tensor": mma_flops / (k2 / 1e3) / 1e12 / peaks.get("bf16_tflops", 1963.0),
        "fp32_equivalent_tflops": algo162 / (k2 / 1e3) / 1e12,
        "wait_errors": bank.wait_errors()}

    # BF16 storage of the score on the same workload (precision form)
    Ub = os3d.new_score(bank, 1, bf16=True)
    fb = torch.empty_like(f)

    def step_bf16():
        os3d.os3d_forward(bank, f, Ub)
        os3d.os3d_inverse(bank, Ub, fb)

    ms_b = timed(step_bf16, args.steps)
    ops["bf16_headline"] = {
        "ms": ms_b, "value": nvox * n_o / (ms_b / 1e3), "unit": UNIT, "udtype": "bf16x2",
        "score_gb": Ub.numel() * Ub.element_size() / 1e9,
        "recon_rel_l2_vs_c64": float(torch.linalg.vector_norm(fb - frec) /
                                     torch.linalg.vector_norm(frec))}
    del Ub, fb
    torch.cuda.empty_cache()
    if world == 1:
        # precision form at 256^3 x 42 and serving, short bounded legs
        ops["precision"] = precision_leg(3, 3)
        ops["serving"] = serve_mix(300, 0.8, False)

    fp32_peak_step = (torch.cuda.get_device_properties(local).multi_processor_count * 128 * 2 *
                      (clk["sm_mhz"] if clk else 2070.0) * 1e6 / 1e12)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, fo, desc, cores = oracle_on_cores(WORKLOAD)
        fg = frec[0].cpu().numpy().astype(np.float64)
        v1, _, desc1, cores1 = oracle_on_cores("tubes32_no42")
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "gpu_recon_rel_l2_vs_oracle": float(np.linalg.norm(fg - fo) / np.linalg.norm(fo)),
               "tubes32_no42": {"value": v1, "unit": UNIT, "cores": cores1, "sample": desc1}}
        try:
            v3, desc3, cores3 = oracle_sample_on_cores("splines256_no42")
            cpu["splines256_no42"] = {"value": v3, "unit": UNIT, "cores": cores3, "sample": desc3}
        except (OSError, MemoryError) as e:   # e.g. no room in the shared-memory file system
            cpu["splines256_no42"] = {"unavailable": f"{type(e).__name__}: {e}"}

    if rank == 0:
        lat = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(dims, n_o, w["L"], "bf16x2" if args.bf16 else "c64", world),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "roofline": roof,
            "step_hbm": {"bytes": step_bytes, "achieved_gbs": step_bytes / (total_ms / args.steps / 1e3) / 1e9},
            "step_alu": {"flops": step_flops,
                         "achieved_tflops": step_flops / (total_ms / args.steps / 1e3) / 1e12,
                         "peak_tflops": fp32_peak_step,
                         "frac": step_flops / (total_ms / args.steps / 1e3) / 1e12 / fp32_peak_step,
                         "peak_kind": "FP32 CUDA-core FMA rate: SMs x 128 lanes x 2 x median SM clock"},
            "kernels": kernels,
            "ops": ops,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nvox * 4,
                    "d2h_bytes_per_step": nvox * 4},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# serving: mixed sizes and orientation counts, Poisson arrivals
# ---------------------------------------------------------------------------
SERVE_SHAPES = [(48, 48, 48), (64, 64, 64), (96, 96, 96), (128, 128, 128), (96, 128, 160)]
SERVE_SUBDIVS = [1, 2]   # 42 or 162 orientations


def run_serve(args):
    import torch
    from paper_1505_07690_gb300 import build
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    build.build()
    print(json.dumps(serve_mix(args.serve, args.load, args.bf16, seed=rank)), flush=True)
    return 0


def serve_mix(n_requests, load, bf16, seed=0):
    """``n_requests`` requests of the mixed workload through the server: first
    all queued at once (capacity), then Poisson arrivals at ``load`` x that
    capacity; p50/p99 latency of the second run."""
    import numpy as np
    import torch
    from paper_1505_07690_gb300 import os3d, synth
    rng = np.random.default_rng(seed)
    # volume pool: 2 seeded spline-tube volumes per shape (volume seed 1000 + k)
    pool = {sh: [torch.from_numpy(synth.spline_tubes(sh, 6, seed=1000 + k, noise=0.2)).pin_memory()
                 for k in range(2)] for sh in SERVE_SHAPES}
    reqs = [(SERVE_SHAPES[rng.integers(len(SERVE_SHAPES))], SERVE_SUBDIVS[rng.integers(2)],
             int(rng.integers(2))) for _ in range(n_requests)]
    n_o = {1: 42, 2: 162}
    vo = [int(np.prod(sh)) * n_o[sd] for sh, sd, _ in reqs]
    srv = os3d.Server(os3d.os3d_server_default_config(arena_bytes=24 << 30, max_inflight=4,
                                                      udtype=1 if bf16 else 0),
                      os3d.os3d_default_params(L=16))

    def drain(outstanding, lat, block):
        while outstanding:
            try:
                _, l = srv.wait(outstanding[0], 600.0 if block else 0.0)
            except os3d.OS3DError as e:
                if e.status == 4:
                    return
                raise
            lat.append(l)
            outstanding.pop(0)

    # banks for every (shape, orientation set), outside the timed part
    warm = [srv.submit(pool[sh][0], sd) for sh in SERVE_SHAPES for sd in SERVE_SUBDIVS]
    for t in warm:
        srv.wait(t, 600.0)
    # capacity: all requests queued at once (closed loop)
    t0 = time.perf_counter()
    out, lat = [], []
    for sh, sd, k in reqs:
        out.append(srv.submit(pool[sh][k], sd))
        drain(out, lat, False)
    drain(out, lat, True)
    t_cap = time.perf_counter() - t0
    capacity = len(reqs) / t_cap
    # Poisson arrivals at load x capacity
    done0, cap0, rep0 = srv.stats()
    rate = load * capacity
    gaps = rng.exponential(1.0 / rate, len(reqs))
    out, lat = [], []
    t0 = time.perf_counter()
    t_next = t0
    for (sh, sd, k), g in zip(reqs, gaps):
        t_next += g
        while time.perf_counter() < t_next:
            drain(out, lat, False)
            time.sleep(min(2e-4, max(0.0, t_next - time.perf_counter())))
        out.append(srv.submit(pool[sh][k], sd))
    drain(out, lat, True)
    t_run = time.perf_counter() - t0
    done, captured, replayed = srv.stats()
    srv.close()
    torch.cuda.empty_cache()
    line = {
        "metric": "serving: forward+inverse per request, mixed sizes, Poisson arrivals; p50/p99 latency",
        "value": sum(vo) / t_run, "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(np.mean(lat))},
        "requests": len(reqs), "requests_per_s": len(reqs) / t_run,
        "capacity_requests_per_s": capacity, "load": load,
        "graphs": {"captured": captured, "replays": replayed, "completed": done,
                   "poisson_run": {"requests": done - done0, "captured": captured - cap0,
                                   "replays": replayed - rep0,
                                   "replay_fraction": (replayed - rep0) / max(done - done0, 1)}},
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serve_mix", "shapes": SERVE_SHAPES, "n_o": [42, 162], "L": 16,
                   "arrival": "poisson", "udtype": "bf16x2" if bf16 else "c64",
                   "max_inflight": 4, "arena_gb": 24},
    }
    return line


# ---------------------------------------------------------------------------
# precision form: complex64 and BF16 storage of U against the exact result
# ---------------------------------------------------------------------------
def run_precision(args):
    from paper_1505_07690_gb300 import build
    build.build()
    line = precision_leg(args.steps, args.warmup)
    if not args.no_cpu_baseline:
        v, _, desc, cores = oracle_on_cores("splines256_no42")
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc}
    print(json.dumps(line), flush=True)
    return 0


def precision_leg(steps, warmup):
    """256^3, 40 spline tubes, 42 orientations, L = 20. For each storage
    format: the relative L2 error of W^-1 W f against the exactly known
    IDFT[1_ball f_hat] (numpy FP64), and of the BF16 score against the
    complex64 one; plus the forward+inverse time of each format."""
    import numpy as np
    import torch
    from paper_1505_07690_gb300 import os3d, synth
    name = "splines256_no42"
    w = synth.WORKLOADS[name]
    dims = w["shape"]
    f_np = synth.workload_volume(name)
    fh = np.fft.fftn(f_np.astype(np.float64))
    k = [np.fft.fftfreq(n) * 2 * np.pi for n in dims]
    r2 = k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2
    fb = np.fft.ifftn(fh * (r2 < np.pi ** 2)).real
    V = os3d.os3d_icosa_orientations(w["subdiv"])
    bank = os3d.os3d_make_wavelets(dims, V, os3d.os3d_default_params(L=w["L"]))
    f = torch.from_numpy(f_np).cuda()
    out = {}
    Uc = None
    for fmt in ("c64", "bf16"):
        U = os3d.new_score(bank, 1, bf16=(fmt == "bf16"))
        fr = torch.empty_like(f)
        for _ in range(max(warmup, 3)):
            os3d.os3d_forward(bank, f, U)
            os3d.os3d_inverse(bank, U, fr)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            os3d.os3d_forward(bank, f, U)
            os3d.os3d_inverse(bank, U, fr)
        b.record()
        torch.cuda.synchronize()
        err = float(np.linalg.norm(fr.cpu().numpy() - fb) / np.linalg.norm(fb))
        rec = {"recon_rel_l2_vs_exact": err, "ms_per_fwd_inv": a.elapsed_time(b) / steps,
               "score_gb": U.numel() * U.element_size() / 1e9}
        if fmt == "c64":
            Uc = U[0, :4].clone()
        else:
            Ub = torch.view_as_complex(U[0, :4].float().contiguous())
            rec["score_rel_l2_vs_c64"] = float(torch.linalg.vector_norm(Ub - Uc) /
                                               torch.linalg.vector_norm(Uc))
        out[fmt] = rec
        del U
        torch.cuda.empty_cache()
    line = {"metric": "precision form: relative L2 error of the reconstruction per score format",
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": name, "dims": list(dims), "n_o": len(V), "L": w["L"]},
            "formats": out, "steps": steps, "warmup": warmup}
    del f, bank
    torch.cuda.empty_cache()
    return line


def run_only_op(args):
    """One operation alone, W warm-up and K timed calls, CUDA events."""
    import numpy as np
    import torch
    from paper_1505_07690_gb300 import build, os3d, synth
    build.build()
    if args.only_op in ("autograd", "score_energy"):
        def timed(fn, n):
            for _ in range(max(args.warmup, 1)):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(n):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / n
    if args.only_op == "autograd":
        r = _autograd_step(os3d, synth, 2 * args.steps, timed)
        print(json.dumps({"op": "autograd", "workload": "splines96x8_no42", **r}), flush=True)
        return 0
    if args.only_op == "score_energy":
        # the one-sweep loss and gradient on the first 2 volumes of the
        # differentiation workload (weights 297 MB, larger than L2)
        w = synth.WORKLOADS["splines96x8_no42"]
        dims = w["shape"]
        V = os3d.os3d_icosa_orientations(w["subdiv"])
        bank = os3d.os3d_make_wavelets(dims, V, os3d.os3d_default_params(L=w["L"]))
        f = torch.from_numpy(np.stack([synth.workload_volume("splines96x8_no42", batch_index=b)
                                       for b in range(2)])).cuda()
        wt = torch.from_numpy(synth.score_weights((8, len(V)) + tuple(dims), seed=1)[:2].copy()).cuda()
        g = torch.empty_like(f)
        scratch = torch.empty(os3d.os3d_score_energy_scratch(bank, 2), dtype=torch.float64,
                              device="cuda")
        ms = timed(lambda: os3d.os3d_score_energy_grad(bank, f, wt, grad_f=g, scratch=scratch),
                   args.steps)
        print(json.dumps({"op": "score_energy", "workload": "splines96x8_no42[:2]", "n_o": len(V),
                          "ms": ms, "steps": args.steps, "loss": float(scratch[0].item())}),
              flush=True)
        return 0
    w = synth.WORKLOADS[WORKLOAD]
    dims = w["shape"]
    V = os3d.os3d_icosa_orientations(w["subdiv"])
    bank = os3d.os3d_make_wavelets(dims, V, os3d.os3d_default_params(L=w["L"]))
    f = torch.from_numpy(synth.workload_volume(WORKLOAD)).cuda()
    fu = torch.empty_like(f)
    dif = os3d.os3d_default_diffusion()
    if args.only_op == "upsilon":
        op = lambda: os3d.os3d_upsilon(bank, f, 1.5, fu)
    elif args.only_op == "enhance_linear_42":
        # the flows of Sec. 4.1 with 42 orientations on the same grid (CUDA cores)
        V = os3d.os3d_icosa_orientations(1)
        bank = os3d.os3d_make_wavelets(dims, V, os3d.os3d_default_params(L=w["L"]))
        op = lambda: os3d.os3d_enhance_linear(bank, f, dif, fu)
    else:
        op = lambda: os3d.os3d_enhance_linear(bank, f, dif, fu)
    for _ in range(max(args.warmup, 1)):
        op()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        op()
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"op": args.only_op, "workload": WORKLOAD, "n_o": len(V),
                      "ms": a.elapsed_time(b) / args.steps, "steps": args.steps,
                      "wait_errors": bank.wait_errors()}), flush=True)
    return 0


def main():
    global WORKLOAD
    args = _args()
    WORKLOAD = args.workload
    if args.impl == "reference":
        return run_reference(args)
    if args.only_op:
        return run_only_op(args)
    if args.serve:
        return run_serve(args)
    if args.precision:
        return run_precision(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
