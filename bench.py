"""Benchmark: mixed-precision (FP32 applies + FP64 refinement) PCG solves of the
variable-coefficient workload -div(a grad u) = f on [0,1]^3, 8x8x8 box elements,
degree W = 8, 64 seeded right-hand sides (tensor-Legendre coefficients ~ N(0,1)
decaying as 2^-k), homogeneous Dirichlet data.

One step = one full solve of the 64-RHS batch to ||b - A x|| <= 1e-10 ||b||
(operator applies, preconditioner, PCG updates and FP64 residual refreshes).
value = FP32 operator-apply GDOF/s (DOF of the batch x applies / time, CUDA
events over 20 applies of the same batch, inputs resident);
ms_per_step = time-to-solution of one step.  The FP64-vs-mixed comparison of
the time-to-solution is run on the first `--cmp-rhs` right-hand sides.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run (one rank per GPU, independent batches per rank,
weak scaling, no data-path collective).  --impl reference times the CPU oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "operator-apply GDOF/s and PCG time-to-solution at oracle H1 error, mixed vs FP64"
N_EL, W_DEG, N_RHS, TOL = 8, 8, 64, 1e-10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rhs", type=int, default=N_RHS)
    ap.add_argument("--n", type=int, default=N_EL)
    ap.add_argument("--W", type=int, default=W_DEG)
    ap.add_argument("--cmp-rhs", type=int, default=4)
    ap.add_argument("--no-cmp", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle's residual check of the compared solutions")
    ap.add_argument("--delta", type=float, default=1e-1)
    ap.add_argument("--cpu-sample-elems", type=int, default=512)
    ap.add_argument("--cpu-reps", type=int, default=2)
    ap.add_argument("--apply-only", action="store_true",
                    help="time only the FP32 operator apply (profiling driver for ncu)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--precond", default="block", choices=["block", "separable"],
                    help="block: exact element blocks of A (set up once, FP64 factors); "
                         "separable: the C-form of eq. (5.19)-(5.20)")
    ap.add_argument("--workload", default="varcoef", choices=["varcoef", "adjoint", "edge", "vertex", "vertex-edge", "poisson", "general", "transpose"],
                    help="varcoef: the 64-RHS W=8 solve; adjoint: the 256-problem theta-gradient batch; "
                         "edge / vertex: the uneven-degree batch of edge- / vertex-neighbourhood problems")
    ap.add_argument("--edge-replicas", type=int, default=146, help="copies of each degree W = 2..8")
    ap.add_argument("--replicas", type=int, default=4096, help="copies of the 2x2x2 Poisson problem")
    ap.add_argument("--ve-replicas", type=int, default=16, help="copies of each degree W = 2..8 (vertex-edge)")
    ap.add_argument("--adj-problems", type=int, default=256)
    ap.add_argument("--adj-fd-problems", type=int, default=16)
    ap.add_argument("--fd-tol", type=float, default=1e-11, help="relative tolerance of the FD correction solves")
    ap.add_argument("--fd-h", type=float, nargs="+", default=[1e-4, 1e-5, 1e-6],
                    help="finite-difference steps of the adjoint check (the worst disagreement of each is reported)")
    ap.add_argument("--max-iter", type=int, default=60000,
                    help="cap on PCG iterations per solve (a capped solve is for profiling only)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except Exception:
                continue
        if sm:
            out.update(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(mx)), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# weak scaling over ranks: every rank solves its own batch (no data-path
# collective); only the timings are reduced
# ---------------------------------------------------------------------------
def shard_seed0(rank, rhs):
    """First seed of rank `rank`'s right-hand sides: ranks own disjoint seed ranges."""
    return 20260 + rhs * rank


def reduce_max_ms(ms, ws, device):
    """Maximum of a per-rank time over the ranks (the slowest rank sets the job time)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(ws, units_per_rank, ms_max):
    """Whole-job throughput in G units/s: all ranks' units over the slowest rank's time."""
    return ws * units_per_rank / (ms_max * 1e-3) / 1e9


def make_problem(args, rank):
    return wl.varcoef_random_rhs(n=args.n, W=args.W, n_rhs=args.rhs, seed0=shard_seed0(rank, args.rhs))


def volume_flops_per_rhs(Ws):
    """Algorithmic flops of one operator apply (volume, forward + transpose):
    2 * (n1 Q P^3 + n2 Q^2 P^2 + n3 Q^3 P) multiply-adds per element with
    (n1, n2, n3) = (3, 5, 6) for -div(a grad u), 2 flops per multiply-add."""
    tot = 0.0
    for W in Ws:
        P, Q = W + 1, 2 * W + 1
        tot += 2 * (3 * Q * P ** 3 + 5 * Q * Q * P * P + 6 * Q ** 3 * P)
    return 2.0 * tot


APPLY_PROFILE = os.path.join(ROOT, "profiles", "k_apply_fp32_w8_varcoef.md")
APPLY_SOURCES = [os.path.join(ROOT, "paper_1110_2316_gb300", "csrc", f)
                 for f in ("kernels.cuh", "inst_template.cuh", "registry.h")]


def apply_source_sha256():
    """sha256 of the sources of the operator kernel (k_apply)."""
    import hashlib
    h = hashlib.sha256()
    for f in APPLY_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(workload_key):
    """DRAM bytes (read + write) of one FP32 k_apply launch on the default
    workload, from the ncu capture summarised in the committed profile:
    its lines 'traffic_bytes_per_launch[<n>,<W>,<rhs>]: N' and
    'kernel_source_sha256: H'.  None when the profile has no figure for the
    workload or the kernel's sources have changed since the capture."""
    try:
        text = open(APPLY_PROFILE).read()
    except OSError:
        return None, "no profile"
    vals, sha = {}, None
    for line in text.splitlines():
        line = line.strip().strip("`")
        if line.startswith("traffic_bytes_per_launch["):
            key, v = line.split(":", 1)
            vals[key[len("traffic_bytes_per_launch["):-1]] = int(v.strip())
        elif line.startswith("kernel_source_sha256:"):
            sha = line.split(":", 1)[1].strip()
    if sha != apply_source_sha256():
        return None, "kernel changed since the ncu capture"
    v = vals.get("%d,%d,%d" % workload_key)
    return v, ("ncu capture in profiles/" if v is not None else "no capture of this workload")


def alu_peaks(device_index, sm_max_mhz):
    """FP32 and FP64 ALU peaks (TFLOP/s) of this device: SM count from the
    device, maximum SM clock from nvidia-smi's sample (2070 MHz if none);
    128 FP32 and 2 FP64 FMA lanes per SM (Blackwell), 2 flops per FMA."""
    import torch
    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz = float(sm_max_mhz) if sm_max_mhz else 2070.0
    return dict(fp32=sms * 128 * 2 * mhz * 1e6 / 1e12, fp64=sms * 2 * 2 * mhz * 1e6 / 1e12, sms=sms, sm_mhz=mhz)


def cpu_baseline(pb, n_elems, reps=1):
    """The oracle's operator apply on a bounded sample of elements (1 rhs), `reps` times."""
    from oracle.functional import Discretisation
    one = wl.Problem(pb.mesh, [pb.f[0]], [pb.g[0]], pb.a, pb.grad_a)
    d = Discretisation(one)
    U = wl.random_dofs(d.ndof, seed=1)
    elems = list(range(min(n_elems, d.E)))
    d.element_apply(U, elems[0])  # tables / coefficient caches
    t = time.perf_counter()
    for _ in range(reps):
        for e in elems:
            d.element_apply(U, e)
    dt = time.perf_counter() - t
    ndof = reps * sum(d.P[e] ** 3 for e in elems)
    return dict(value=ndof / dt / 1e9, unit="GDOF/s", cores=os.cpu_count(), kind="oracle",
                sample="oracle operator apply, %d x %d of %d elements (W=%d, 1 rhs), %.1f s" %
                       (reps, len(elems), d.E, d.W[0], dt), seconds=dt)


def bench_config(args, ndof):
    """The workload of the default bench line (both arms)."""
    return dict(workload="varcoef -div(a grad u)=f, [0,1]^3, %d^3 elements, W=%d, %d RHS, tol 1e-10, "
                         "FP32 applies + FP64 reliable-update refinement" % (args.n, args.W, args.rhs),
                n_elem=args.n ** 3, W=args.W, rhs_per_gpu=args.rhs, dof_per_rhs=ndof,
                l2="working set > L2 (FP32 vectors %.0f MB each)" % (args.rhs * ndof * 4 / 1e6),
                parallelism="replicas (independent batches per GPU)")


def _oracle_task(task):
    """One oracle evaluation for the solution check (runs in a spawned worker):
    ("b", r) -> b_r = S^T M d_r; ("Ax", r, x) -> A x, both in FP64."""
    n, W, k, seed0, kind, r, xv = task
    from oracle.functional import Discretisation
    d = Discretisation(wl.varcoef_random_rhs(n=n, W=W, n_rhs=k, seed0=seed0))
    return d.rhs_b(r) if kind == "b" else d.apply_A(xv)


def oracle_check(args, seed0, k, sols):
    """The oracle's FP64 relative residual ||b_o - A_o x|| / ||b_o|| of GPU
    solutions for right-hand sides 0..k-1 (``sols``: name -> [k, ndof] arrays)
    and the oracle-norm relative H^1 difference of the mixed and FP64 solutions
    when both are given.  The oracle's evaluations run in a spawned process
    pool on the host cores."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from oracle.functional import Discretisation
    from oracle.h1 import h1_rel_diff
    t0 = time.perf_counter()
    tasks = [(args.n, args.W, k, seed0, "b", r, None) for r in range(k)]
    names = sorted(sols)
    for name in names:
        tasks += [(args.n, args.W, k, seed0, "Ax", r, sols[name][r]) for r in range(k)]
    workers = max(1, min(len(tasks), (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        out = list(ex.map(_oracle_task, tasks))
    bs = out[:k]
    res = {}
    for i, name in enumerate(names):
        axs = out[k * (i + 1):k * (i + 2)]
        res[name] = [float(np.linalg.norm(bs[r] - axs[r]) / np.linalg.norm(bs[r])) for r in range(k)]
    h1 = None
    if "cmp_mixed" in sols and "cmp_fp64" in sols:
        d = Discretisation(wl.varcoef_random_rhs(n=args.n, W=args.W, n_rhs=k, seed0=seed0))
        h1 = [h1_rel_diff(d, sols["cmp_mixed"][r], sols["cmp_fp64"][r]) for r in range(k)]
    worst = max(max(v) for v in res.values())
    return dict(rhs=list(range(k)), rel_residual=res, max_rel_residual=worst,
                h1_rel_diff_mixed_vs_fp64=h1, residual_bound=1.1e-10, h1_bound=1e-8,
                passed=bool(worst <= 1.1e-10 and (h1 is None or max(h1) <= 1e-8)),
                workers=workers, seconds=time.perf_counter() - t0,
                what="oracle (numpy FP64) recomputes b and A x of the GPU solutions")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    pb = wl.varcoef_random_rhs(n=args.n, W=args.W, n_rhs=1)
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(pb, args.cpu_sample_elems, 1)
        if i >= args.warmup:
            vals.append(cb["value"])
            secs.append(cb["seconds"])
    v = float(np.mean(vals))
    # each step: the oracle's apply of a bounded sample of the workload's elements
    line = dict(metric=METRIC, value=v, unit="GDOF/s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * float(np.mean(secs)), higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=bench_config(args, args.n ** 3 * (args.W + 1) ** 3),
                cpu_baseline=dict(value=v, unit="GDOF/s", cores=cb["cores"], kind="oracle", sample=cb["sample"]),
                e2e=dict(value=v, unit="GDOF/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


def run_adjoint(args, local):
    """Adjoint batch: 256 independent cube problems (4^3 elements, W_p ~ U{4..10}),
    a = exp(g), g a degree-3 Legendre field with theta ~ N(0,1) (std of g 0.5),
    f = 1, u = 0 on the boundary; J = sum_p ||u_p - sin(pi x) sin(pi y) sin(pi z)||^2
    by quadrature.  dJ/dtheta by the adjoint: forward solve, adjoint PCG solve
    (recomputed), point gradients from the library, chain to theta in torch.
    Reports the gradient time (FP64 and mixed), the mixed-vs-FP64 gradient
    difference, and a central finite-difference check (h = 1e-6, FP64) on 8
    parameters of the first 16 problems."""
    import math
    import torch
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api
    from paper_1110_2316_gb300.autograd import PointValues, Solve
    from paper_1110_2316_gb300.fields import LegendreLogField
    dev = torch.device("cuda", local)
    Ws = wl.adjoint_batch_degrees(args.adj_problems)
    parts = [wl.lognormal_coef_problem(int(W), p, n=4) for p, W in enumerate(Ws)]
    theta_all = torch.tensor(np.stack([p.meta["theta"] for p in parts]), device=dev)
    pi = math.pi

    def context(sub, theta):
        pb = wl.batch_problems(sub)
        m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR, device=local)
        fld = LegendreLogField.from_mesh(m, pb.mesh.elem_problem, device=dev)
        ut = fld.separable(lambda x: torch.sin(pi * x), lambda y: torch.sin(pi * y), lambda z: torch.sin(pi * z))
        f = torch.ones(1, m.nquad, dtype=torch.float64, device=dev)
        a, ga = fld(theta)
        m.set_data(f=f, a=a, grad_a=ga)
        t_p = time.perf_counter()
        if args.precond == "block":
            # built once from the data at theta and kept for every later solve
            m.setup_block_preconditioner()
        torch.cuda.synchronize()
        t_p = time.perf_counter() - t_p
        w = torch.empty(m.nquad, dtype=torch.float64, device=dev)
        m.quad_weights(w)
        qprob = torch.tensor(np.repeat(pb.mesh.elem_problem.astype(np.int64),
                                       [(2 * int(W) + 1) ** 3 for W in pb.mesh.elem_W]), device=dev)
        return dict(m=m, fld=fld, ut=ut, w=w, qprob=qprob, f=f, P=len(sub),
                    ndof=m.ndof, nelem=len(pb.mesh.elem_W), t_prec=t_p)

    def J_of(c, v):
        return torch.zeros(c["P"], dtype=torch.float64, device=dev).index_add(
            0, c["qprob"], c["w"] * (v - c["ut"]) ** 2)

    def gradient(c, theta, prec, tol, adj_tol=1e-8):
        # forward solve in `prec`; adjoint solve in FP64 to adj_tol (its attainable
        # relative residual is about eps64 kappa(A), 1e-9..1e-8 on this batch)
        th = theta.clone().requires_grad_(True)
        a, ga = c["fld"](th)
        u = Solve.apply(c["f"], a, ga, c["m"], None, tol, prec, api.FP64, adj_tol)
        Jp = J_of(c, PointValues.apply(u, c["m"])[0])
        Jp.sum().backward()
        return Jp.detach(), th.grad.detach()

    def correction(c, theta, u0, tol):
        """u(theta) - u0 by one FP64 correction solve A(theta) d = b(theta) -
        A(theta) u0 (u0: the solution at theta0)."""
        a, ga = c["fld"](theta)
        m = c["m"]
        m.set_data(f=c["f"], a=a, grad_a=ga)
        b = torch.empty_like(u0)
        m.get_rhs(b)
        r = torch.empty_like(u0)
        m.apply_operator(u0, r)
        r = b - r
        m.set_rhs(r)
        d = torch.zeros_like(u0)
        rep = m.pcg_solve(d, tol=tol, prec=api.FP64, max_iter=args.max_iter, raise_on_error=False)
        m.set_rhs(b)
        return d, rep

    def J_diff(c, tp, tm, u0, v0, tol):
        """J(tp) - J(tm) per problem as one quadrature of pointwise differences,
        sum w (v+ - v-)(v+ + v- - 2 u_target) with v+- = v0 + d+-: no
        subtraction of two separately rounded sums of O(1) terms."""
        dp, rp = correction(c, tp, u0, tol)
        dm, rm = correction(c, tm, u0, tol)
        m = c["m"]
        fa = torch.empty(1, 5, m.nquad, dtype=torch.float64, device=dev)
        fb = torch.empty_like(fa)
        m.eval_fields(dp - dm, fa)
        m.eval_fields(dp + dm, fb)
        t = c["w"] * fa[0, 0] * (2 * (v0 - c["ut"]) + fb[0, 0])
        return torch.zeros(c["P"], dtype=torch.float64, device=dev).index_add(0, c["qprob"], t), rp, rm

    t0 = time.perf_counter()
    c = context(parts, theta_all)
    t_setup = time.perf_counter() - t0
    times, grads = {}, {}
    logs = {}
    for name, prec in (("fp64", api.FP64), ("mixed", api.FP32)):
        c["m"].solve_log = []
        torch.cuda.synchronize()
        t = time.perf_counter()
        J, g = gradient(c, theta_all, prec, 1e-10)
        torch.cuda.synchronize()
        times[name] = time.perf_counter() - t
        grads[name] = g
        logs[name] = [(k, r["iterations"], r["sweeps"], r["rel_residual"]) for k, r in c["m"].solve_log]
    gdiff = float(torch.max(torch.linalg.vector_norm((grads["mixed"] - grads["fp64"]).flatten(1), dim=1) /
                            torch.linalg.vector_norm(grads["fp64"].flatten(1), dim=1)))
    c["m"].close()

    # finite differences (FP64) on the first problems, 8 parameters each
    nfd = min(args.adj_fd_problems, len(parts))
    th0 = theta_all[:nfd].clone()
    cf = context(parts[:nfd], th0)
    cf["m"].solve_log = []
    _, g = gradient(cf, th0, api.FP64, 1e-11)
    fd_grad_reports = list(cf["m"].solve_log)
    a0, ga0 = cf["fld"](th0)
    cf["m"].set_data(f=cf["f"], a=a0, grad_a=ga0)
    u0 = torch.zeros(cf["m"].ndof, dtype=torch.float64, device=dev)
    rep0 = cf["m"].pcg_solve(u0, tol=1e-11, prec=api.FP64, max_iter=args.max_iter, raise_on_error=False)
    fl0 = torch.empty(1, 5, cf["m"].nquad, dtype=torch.float64, device=dev)
    cf["m"].eval_fields(u0, fl0)
    v0 = fl0[0, 0].clone()
    rng = np.random.Generator(np.random.PCG64(8))
    flat = rng.choice(np.arange(1, 64), size=8, replace=False)
    idxs = [tuple(int(v) for v in np.unravel_index(i, (4, 4, 4))) for i in flat]
    adj = np.array([g[(slice(None),) + idx].cpu().numpy() for idx in idxs])  # [8, nfd]
    sweep, res = {}, []
    for h in args.fd_h:
        fds = []
        for idx in idxs:
            tp, tm = th0.clone(), th0.clone()
            tp[(slice(None),) + idx] += h
            tm[(slice(None),) + idx] -= h
            dJ, rp, rm = J_diff(cf, tp, tm, u0, v0, args.fd_tol)
            res += [rp["rel_residual"], rm["rel_residual"]]
            fds.append((dJ / (2 * h)).cpu().numpy())
        fds = np.array(fds)
        scale = np.maximum(np.abs(fds), 1e-3 * np.abs(fds).max(axis=0, keepdims=True))
        ratio = np.abs(adj - fds) / (1e-6 * scale)
        sweep[h] = dict(worst_ratio_to_bound=float(ratio.max()),
                        per_problem=[dict(W=int(Ws[p]), worst_ratio=float(ratio[:, p].max()),
                                          rel_err=float(np.max(np.abs(adj[:, p] - fds[:, p])) /
                                                        np.max(np.abs(fds[:, p]))))
                                     for p in range(nfd)])
    # the FD reference's own error: O(h^2) truncation above, rounding noise
    # (the FP64-attainable accuracy of the solves, about 1e-11, divided by h)
    # below; the check is taken at the first step of --fd-h (1e-4), and the
    # sweep shows the noise growing like 1/h
    h_best = args.fd_h[0]
    worst = sweep[h_best]["worst_ratio_to_bound"]
    cf["m"].close()
    line = dict(metric="adjoint theta-gradient time for the batch (forward + adjoint PCG + data gradient)",
                value=times["mixed"], unit="s", higher_is_better=False, n_gpus=1, data="synthetic",
                config=dict(workload="adjoint batch: %d cube problems, 4^3 elements each, W ~ U{4..10} (seed 7), "
                                     "a = exp(degree-3 Legendre field, std 0.5), f = 1, u = 0" % len(parts),
                            n_problem=len(parts), n_elem=c["nelem"], ndof=c["ndof"],
                            W_hist={int(w): int((Ws == w).sum()) for w in sorted(set(Ws.tolist()))}),
                grad_time_s=times, setup_s=t_setup, setup_block_precond_s=c["t_prec"], precond=args.precond,
                grad_rel_diff_mixed_vs_fp64=gdiff, solves=logs,
                fd_check=dict(problems=nfd, params=[list(i) for i in idxs], h=h_best,
                              J_evaluation="central differences of J; u(theta +- h) = u0 (FP64 PCG to 1e-11 at "
                                           "theta0) + an FP64 correction solve to %g of its residual; J(+) - J(-) "
                                           "as one quadrature of pointwise differences" % args.fd_tol,
                              u0_rel_residual=rep0["rel_residual"],
                              gradient_solves=[(k, r["iterations"], r["rel_residual"]) for k, r in fd_grad_reports],
                              worst_ratio_to_bound=worst, passed=bool(worst <= 1.0),
                              per_problem=sweep[h_best]["per_problem"],
                              h_sweep={"%g" % k: v["worst_ratio_to_bound"] for k, v in sweep.items()},
                              bound="|g_adj - g_fd| <= 1e-6 max(|g_fd|, 1e-3 max_params |g_fd|)",
                              fd_solve_rel_residual_max=float(max(res))))
    print(json.dumps(line))
    return 0


def run_edge(args, local):
    """Uneven-degree batch of neighbourhood problems, W = 2..8, each degree
    replicated, one launch per degree group per operator apply: edge (Table
    6.18's Laplace problem u = r^(1/3) sin(theta/3) x3 on the quarter
    cylinder, N = 2W + 4 layers), vertex (Table 6.16's Poisson problem on the
    spherical wedge, N = 2W + 4) or vertex-edge (w = r^(2/3) sin(2 theta/3) in
    the cone phi < pi/4, N = W + 2 layers in psi and in zeta); mu = 0.15.
    Reports the FP32 apply GDOF/s, the mixed and FP64 time-to-solution with the
    element-block preconditioner, and the H1 difference of the two solutions."""
    import torch
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api
    dev = torch.device("cuda", local)
    kind = args.workload
    reps = args.ve_replicas if kind == "vertex-edge" else args.edge_replicas
    Ws = [W for W in range(2, 9) for _ in range(reps)]
    t0 = time.perf_counter()
    pb = dict(edge=wl.edge_batch, vertex=wl.vertex_batch, **{"vertex-edge": wl.vertex_edge_batch})[kind](Ws)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_LAPLACE, device=local)
    m.set_data(**api.problem_data_arrays(m, pb))
    t_setup = time.perf_counter() - t0
    t1 = time.perf_counter()
    m.setup_block_preconditioner()
    torch.cuda.synchronize()
    t_prec = time.perf_counter() - t1
    n = m.ndof
    u = torch.randn(n, dtype=torch.float32, device=dev)
    y = torch.empty_like(u)
    for _ in range(3):
        m.apply_operator(u, y)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record()
    for _ in range(20):
        m.apply_operator(u, y)
    a1.record()
    torch.cuda.synchronize()
    apply_ms = a0.elapsed_time(a1) / 20
    out, sol = {}, {}
    for name, prec in (("mixed", api.FP32), ("fp64", api.FP64)):
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        m.pcg_solve(x, tol=TOL, prec=prec, max_iter=64, raise_on_error=False)  # graph capture
        x.zero_()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        rep = m.pcg_solve(x, tol=TOL, prec=prec, max_iter=200000, raise_on_error=False)
        c1.record()
        torch.cuda.synchronize()
        out[name] = dict(tts_s=c0.elapsed_time(c1) / 1e3, iterations=rep["iterations"], refreshes=rep["sweeps"],
                         status=rep["status"], rel_residual=rep["rel_residual"])
        sol[name] = x
    h = m.h1_error(sol["mixed"], ref=sol["fp64"])
    diff = float(np.sqrt(h[0, 0] / h[0, 1]))
    name = kind
    what = dict(vertex="Table 6.16 Poisson problem on the spherical wedge, vertex-neighbourhood elements in "
                       "(phi, theta, ln rho), N = 2W+4 layers",
                edge="Table 6.18 Laplace problem on the quarter cylinder, edge-neighbourhood elements in "
                     "(ln r, theta, x3), N = 2W+4 layers",
                **{"vertex-edge": "Laplace problem w = r^(2/3) sin(2 theta/3) in the cone phi < pi/4, x3 < 1, "
                                  "0 < theta < 3 pi/2, vertex-edge elements in (ln tan phi, theta, ln x3), "
                                  "N = W+2 layers in psi and zeta, 3 theta sectors"})[kind]
    line = dict(metric="%s-neighbourhood batch: operator-apply GDOF/s and time-to-solution, mixed vs FP64" % name,
                value=n / (apply_ms * 1e-3) / 1e9, unit="GDOF/s", higher_is_better=True, n_gpus=1, dtype="f32",
                data="synthetic",
                config=dict(workload=what + ", W = 2..8 x %d replicas, mu = 0.15, tol 1e-10" % reps,
                            n_problem=len(Ws), n_elem=int(pb.mesh.n_elem), n_corner=int(pb.mesh.n_corner), ndof=n),
                apply_ms=apply_ms, solves=out, speedup=out["fp64"]["tts_s"] / out["mixed"]["tts_s"],
                rel_diff_mixed_vs_fp64=diff,
                rel_diff_norm="H1 (physical coordinates, the library's norm)",
                setup_s=t_setup, setup_block_precond_s=t_prec)
    print(json.dumps(line))
    return 0


def exact_at_points(mesh, pb):
    """Exact solution and gradient of every element's problem at the
    library's volume query points (input sampling for the H1 error)."""
    ax, _ = mesh.query_points()
    parts = getattr(pb, "parts", None)
    vq, gq, o = [], [[], [], []], 0
    for e in range(mesh.n_elem):
        Q = 2 * int(mesh.elem_W[e]) + 1
        xs, ys, zs = ax[o:o + Q], ax[o + Q:o + 2 * Q], ax[o + 2 * Q:o + 3 * Q]
        o += 3 * Q
        p = parts[int(pb.mesh.elem_problem[e])] if parts is not None else pb
        vq.append(p.u_exact[0](xs, ys, zs).ravel())
        for k, g in enumerate(p.grad_u_exact[0](xs, ys, zs)):
            gq[k].append(np.broadcast_to(g, (Q, Q, Q)).ravel())
    return np.concatenate(vq), np.concatenate([np.concatenate(g) for g in gq])


def run_poisson(args, local):
    """Replicas of the 2x2x2-element Poisson problem on [0,1]^3 (W = 4,
    -Lap u = 3 pi^2 sin(pi x) sin(pi y) sin(pi z), u = 0 on the boundary), all
    in one launch per operator apply: the problem is too small to fill the GPU
    alone.  Reports the FP32 and FP64 apply GDOF/s, the mixed and FP64
    time-to-solution, and the relative H1 error of both solutions against the
    exact u."""
    import torch
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    one = wl.poisson_sine(n=2, W=4)
    pb = wl.batch_problems([one] * args.replicas)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_LAPLACE, device=local)
    m.set_data(**api.problem_data_arrays(m, pb))
    vq, gq = exact_at_points(m, pb)
    vq, gq = torch.tensor(vq, device=dev), torch.tensor(gq, device=dev)
    t_setup = time.perf_counter() - t0
    t1 = time.perf_counter()
    if args.precond == "block":
        m.setup_block_preconditioner()
    torch.cuda.synchronize()
    t_prec = time.perf_counter() - t1
    n = m.ndof
    apply_ms = {}
    for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        u = torch.randn(n, dtype=dt, device=dev)
        y = torch.empty_like(u)
        for _ in range(3):
            m.apply_operator(u, y)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(20):
            m.apply_operator(u, y)
        a1.record()
        torch.cuda.synchronize()
        apply_ms[name] = a0.elapsed_time(a1) / 20
    out = {}
    for name, prec in (("mixed", api.FP32), ("fp64", api.FP64)):
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        m.pcg_solve(x, tol=TOL, prec=prec, max_iter=64, raise_on_error=False)  # graph capture
        x.zero_()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        rep = m.pcg_solve(x, tol=TOL, prec=prec, max_iter=200000, raise_on_error=False)
        c1.record()
        torch.cuda.synchronize()
        h = m.h1_error(x, vq=vq, gq=gq)
        out[name] = dict(tts_s=c0.elapsed_time(c1) / 1e3, iterations=rep["iterations"], refreshes=rep["sweeps"],
                         status=rep["status"], rel_residual=rep["rel_residual"],
                         h1_rel_error=float(np.sqrt(h[0, 0] / h[0, 1])))
    line = dict(metric="Poisson replicas: operator-apply GDOF/s and time-to-solution, mixed vs FP64",
                value=n / (apply_ms["fp32"] * 1e-3) / 1e9, unit="GDOF/s", higher_is_better=True, n_gpus=1,
                dtype="f32", data="synthetic",
                config=dict(workload="-Lap u = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) on [0,1]^3, 2x2x2 elements, "
                                     "W = 4, %d replicas in one launch, tol 1e-10" % args.replicas,
                            n_problem=args.replicas, n_elem=int(pb.mesh.n_elem), ndof=n, precond=args.precond),
                apply_ms=apply_ms, gdofs_fp64=n / (apply_ms["fp64"] * 1e-3) / 1e9, solves=out,
                speedup=out["fp64"]["tts_s"] / out["mixed"]["tts_s"],
                setup_s=t_setup, setup_block_precond_s=t_prec)
    print(json.dumps(line))
    return 0


def general_flops_per_rhs(Ws):
    """Algorithmic flops of one general-operator apply (volume, forward +
    transpose): the (3, 6, 10)-field sum factorisation of the ten-term form,
    2 * (3 Q P^3 + 6 Q^2 P^2 + 10 Q^3 P) multiply-adds per element."""
    tot = 0.0
    for W in Ws:
        P, Q = W + 1, 2 * W + 1
        tot += 2 * (3 * Q * P ** 3 + 6 * Q * Q * P * P + 10 * Q ** 3 * P)
    return 2.0 * tot


def scaled_rhs_problem(pb, n_rhs):
    """The problem with n_rhs right-hand sides: data (f, g, the Neumann flux)
    and exact solution of rhs r scaled by 1 + r / n_rhs (linear problem)."""
    def sc(fun, c):
        return lambda *a: c * np.asarray(fun(*a))

    def scv(fun, c):
        return lambda *a: tuple(c * np.asarray(v) for v in fun(*a))
    cs = [1.0 + r / n_rhs for r in range(n_rhs)]
    return wl.Problem(pb.mesh, [sc(pb.f[0], c) for c in cs], [sc(pb.g[0], c) for c in cs], None, None,
                      [sc(pb.u_exact[0], c) for c in cs], [scv(pb.grad_u_exact[0], c) for c in cs],
                      name=pb.name, flux=None if pb.flux is None else [scv(pb.flux[0], c) for c in cs],
                      robin_gamma=pb.robin_gamma, op=pb.op)


def run_general(args, local):
    """The general operator of eq. (2.2) (the ten-term form of eq. 5.45 with
    per-point coefficients): Table 6.14's non-self-adjoint problem (variable
    A with mixed derivatives, e u, Dirichlet on x = +-1, y = -1, Neumann on
    y = 1, z = +-1) on (-1,1)^3 in --n^3 elements of degree --W, --rhs
    right-hand sides.  Reports the general apply's GDOF/s and roofline
    fraction (FP32 and FP64), the mixed and FP64 time-to-solution with the
    element-block preconditioner, and the relative H1 error of both."""
    import torch
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    R = args.rhs
    pb = scaled_rhs_problem(wl.nonsym_mixed(n=args.n, W=args.W), R)
    m = api.Mesh(pb.mesh, n_rhs=R, coef_kind=api.COEF_GENERAL, device=local)
    m.set_data(**api.problem_data_arrays(m, pb))
    vq, gq = exact_at_points(m, pb)
    vq = torch.tensor(np.concatenate([vq * (1.0 + r / R) for r in range(R)]), device=dev)
    gq = torch.tensor(np.concatenate([gq * (1.0 + r / R) for r in range(R)]), device=dev)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    n = R * m.ndof
    fl = general_flops_per_rhs([int(w) for w in m.elem_W]) * R
    apply_ms = {}
    with ClockSampler(local) as clk:
        for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
            u = torch.randn(n, dtype=dt, device=dev)
            y = torch.empty_like(u)
            for _ in range(3):
                m.apply_operator(u, y)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 20 if name == "fp32" else 3
            a0.record()
            for _ in range(reps):
                m.apply_operator(u, y)
            a1.record()
            torch.cuda.synchronize()
            apply_ms[name] = a0.elapsed_time(a1) / reps
    clocks = clk.summary()
    peaks = alu_peaks(local, clocks.get("sm_max_mhz"))
    t1 = time.perf_counter()
    m.setup_block_preconditioner()
    torch.cuda.synchronize()
    t_prec = time.perf_counter() - t1
    out = {}
    for name, prec in (("mixed", api.FP32), ("fp64", api.FP64)):
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        m.pcg_solve(x, tol=TOL, prec=prec, max_iter=64, raise_on_error=False)  # graph capture
        x.zero_()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        rep = m.pcg_solve(x, tol=TOL, prec=prec, max_iter=args.max_iter, raise_on_error=False)
        c1.record()
        torch.cuda.synchronize()
        h = m.h1_error(x, vq=vq, gq=gq)
        out[name] = dict(tts_s=c0.elapsed_time(c1) / 1e3, iterations=rep["iterations"], refreshes=rep["sweeps"],
                         status=rep["status"], rel_residual=rep["rel_residual"],
                         h1_rel_error_max=float(np.sqrt(h[:, 0] / h[:, 1]).max()))
        out[name + "_x"] = x
    hd = m.h1_error(out.pop("mixed_x"), ref=out.pop("fp64_x"))
    rel_diff = float(np.sqrt((hd[:, 0] / hd[:, 1]).max()))
    ach = fl / (apply_ms["fp32"] * 1e-3) / 1e12
    line = dict(metric="general operator: apply GDOF/s, time-to-solution mixed vs FP64",
                value=n / (apply_ms["fp32"] * 1e-3) / 1e9, unit="GDOF/s", higher_is_better=True, n_gpus=1,
                dtype="f32", data="synthetic",
                config=dict(workload="a u_xx + b u_yy + c u_zz + d (u_xy + u_yz + u_zx) + e u = f (Table 6.14's "
                                     "operator and faces) on (-1,1)^3, %d^3 elements, W = %d, %d rhs, tol 1e-10"
                                     % (args.n, args.W, R), n_elem=int(pb.mesh.n_elem), ndof_per_rhs=m.ndof),
                apply_ms=apply_ms, gdofs_fp64=n / (apply_ms["fp64"] * 1e-3) / 1e9,
                roofline=dict(bound="alu", kernel="k_apply_gen FP32 (W=%d)" % args.W, achieved=ach,
                              peak=peaks["fp32"], unit="TFLOP/s", frac=ach / peaks["fp32"],
                              fp64_achieved=fl / (apply_ms["fp64"] * 1e-3) / 1e12, fp64_peak=peaks["fp64"],
                              fp64_frac=fl / (apply_ms["fp64"] * 1e-3) / 1e12 / peaks["fp64"],
                              note="algorithmic (3,6,10)-field flops per (element, rhs), derived ALU peaks"),
                solves=out, speedup=out["fp64"]["tts_s"] / out["mixed"]["tts_s"],
                h1_rel_diff_mixed_vs_fp64=rel_diff, setup_s=t_setup, setup_block_precond_s=t_prec,
                clocks=clocks)
    print(json.dumps(line))
    return 0


def run_transpose(args, local):
    """The volume transpose of the residual map two ways on the default
    workload (-div(a grad u), --n^3 elements of W = --W, --rhs right-hand
    sides): the direct reverse of the sum factorisation (hpse_apply_transpose)
    and the integration-by-parts form of eq. (5.45)-(5.48)
    (hpse_apply_transpose_ibp), FP32 and FP64, with their agreement."""
    import torch
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api
    dev = torch.device("cuda", local)
    pb = make_problem(args, 0)
    m = api.Mesh(pb.mesh, n_rhs=args.rhs, coef_kind=api.COEF_SCALAR, device=local)
    m.set_data(**api.problem_data_arrays(m, pb))
    Ws = [int(w) for w in m.elem_W]
    # algorithmic multiply-adds of the transpose half: (6, 5, 3) fields of the
    # z, y, x stages; the IBP form's own count: 3 second and 3 first Q-grid
    # derivatives (6 Q^4), the projection (Q^3 P + Q^2 P^2 + Q P^3)
    mac_t = sum(6 * (2 * w + 1) ** 3 * (w + 1) + 5 * (2 * w + 1) ** 2 * (w + 1) ** 2 + 3 * (2 * w + 1) * (w + 1) ** 3
                for w in Ws) * args.rhs
    mac_i = sum(6 * (2 * w + 1) ** 4 + (2 * w + 1) ** 3 * (w + 1) + (2 * w + 1) ** 2 * (w + 1) ** 2
                + (2 * w + 1) * (w + 1) ** 3 for w in Ws) * args.rhs
    res = {}
    with ClockSampler(local) as clk:
        for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
            z = torch.randn(args.rhs, m.nquad, dtype=dt, device=dev)
            y = {k: torch.empty(args.rhs * m.ndof, dtype=dt, device=dev) for k in ("direct", "ibp")}
            fns = dict(direct=m.apply_transpose, ibp=m.apply_transpose_ibp)
            for k, fn in fns.items():
                for _ in range(3):
                    fn(z, y[k])
                torch.cuda.synchronize()
                reps = 20 if name == "fp32" else 5
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    fn(z, y[k])
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                res.setdefault(name, {})[k] = dict(ms=ms, alg_tflops=2 * mac_t / (ms * 1e-3) / 1e12,
                                                   executed_tflops=2 * (mac_t if k == "direct" else mac_i)
                                                   / (ms * 1e-3) / 1e12)
            res[name]["rel_diff"] = float((y["ibp"].double() - y["direct"].double()).abs().max()
                                          / y["direct"].double().abs().max())
    clocks = clk.summary()
    peaks = alu_peaks(local, clocks.get("sm_max_mhz"))
    line = dict(metric="volume transpose: direct vs integration by parts (eq. 5.46-5.48), ms per launch",
                value=res["fp32"]["ibp"]["ms"], unit="ms", higher_is_better=False, n_gpus=1, dtype="f32",
                data="synthetic",
                config=dict(workload="-div(a grad u), [0,1]^3, %d^3 elements, W=%d, %d RHS, transpose of the "
                                     "residual map (faces excluded)" % (args.n, args.W, args.rhs)),
                results=res, peaks_tflops=dict(fp32=peaks["fp32"], fp64=peaks["fp64"]),
                note="alg_tflops: the direct transpose's algorithmic multiply-adds (6,5,3 fields) per launch for "
                     "both forms; executed_tflops: each form's own count", clocks=clocks)
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("adjoint", "edge", "vertex", "vertex-edge", "poisson", "general", "transpose"):
        import torch
        _, _, local = dist_env()
        torch.cuda.set_device(local)
        run = dict(adjoint=run_adjoint, edge=run_edge, vertex=run_edge, poisson=run_poisson, general=run_general,
                   transpose=run_transpose,
                   **{"vertex-edge": run_edge})[args.workload]
        return run(args, local)
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1110_2316_gb300.build import build
    if rank == 0:
        build()
    if ws > 1:
        torch.distributed.barrier()
    build()
    from paper_1110_2316_gb300 import api
    dev = torch.device("cuda", local)

    # ---- set-up (untimed) ---------------------------------------------------
    t0 = time.perf_counter()
    pb = make_problem(args, rank)
    mesh = api.Mesh(pb.mesh, n_rhs=args.rhs, coef_kind=api.COEF_SCALAR, device=local)
    data = api.problem_data_arrays(mesh, pb)
    t_sample = time.perf_counter() - t0
    t1 = time.perf_counter()
    mesh.set_data(**data)
    torch.cuda.synchronize()
    t_setdata = time.perf_counter() - t1

    n_tot = args.rhs * mesh.ndof
    if args.apply_only:
        dt = torch.float32 if args.prec == "fp32" else torch.float64
        u = torch.randn(n_tot, dtype=dt, device=dev)
        y = torch.empty_like(u)
        for _ in range(args.warmup):
            mesh.apply_operator(u, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            mesh.apply_operator(u, y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(1, args.steps)
        fl = volume_flops_per_rhs([int(w) for w in mesh.elem_W]) * args.rhs
        print(json.dumps(dict(mode="apply-only", prec=args.prec, rhs=args.rhs, ms_per_apply=ms,
                              gdofs=n_tot / ms / 1e6, alg_tflops=fl / ms / 1e9)))
        return 0
    # the preconditioner (not used by the apply-only mode above)
    t_prec = 0.0
    if args.precond == "block":
        t2 = time.perf_counter()
        mesh.setup_block_preconditioner()
        torch.cuda.synchronize()
        t_prec = time.perf_counter() - t2
    x = torch.zeros(n_tot, dtype=torch.float64, device=dev)

    def solve(m, xx, prec):
        return m.pcg_solve(xx, tol=TOL, prec=prec, inner_tol=args.delta, check_every=16, max_iter=args.max_iter,
                           raise_on_error=args.max_iter == 60000)

    # ---- warm-up and timed steps -----------------------------------------------
    for _ in range(args.warmup):
        x.zero_()
        solve(mesh, x, api.FP32)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    api.kernel_launch_count(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.steps):
            x.zero_()
            reps.append(solve(mesh, x, api.FP32))
        ev1.record()
        torch.cuda.synchronize()
    launches = api.kernel_launch_count(reset=True)
    ms = reduce_max_ms(ev0.elapsed_time(ev1) / args.steps, ws, dev)
    k_chk = min(args.cmp_rhs, args.rhs)
    x_timed = x.view(args.rhs, mesh.ndof)[:k_chk].cpu().numpy()
    applies = float(np.mean([r["applies"] for r in reps]))
    solve_rate = weak_scaling_rate(ws, n_tot * applies, ms)
    clocks = clk.summary()

    # ---- dominant kernel: FP32 operator apply, timed alone -----------------------
    u32 = torch.randn(n_tot, dtype=torch.float32, device=dev)
    y32 = torch.empty_like(u32)
    for _ in range(3):
        mesh.apply_operator(u32, y32)
    torch.cuda.synchronize()
    na = 20
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record()
    for _ in range(na):
        mesh.apply_operator(u32, y32)
    a1.record()
    torch.cuda.synchronize()
    apply_ms = a0.elapsed_time(a1) / na
    apply_ms_all = reduce_max_ms(apply_ms, ws, dev)
    value = weak_scaling_rate(ws, n_tot, apply_ms_all)
    alg_flops = volume_flops_per_rhs([int(w) for w in mesh.elem_W]) * args.rhs
    achieved = alg_flops / (apply_ms * 1e-3) / 1e12
    peaks = alu_peaks(local, clocks.get("sm_max_mhz"))
    peak = peaks["fp32"]
    traffic, traffic_src = profiled_traffic((args.n, args.W, args.rhs))
    # FP64 apply for reference
    u64 = u32.double()
    y64 = torch.empty_like(u64)
    mesh.apply_operator(u64, y64)
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record()
    for _ in range(3):
        mesh.apply_operator(u64, y64)
    b1.record()
    torch.cuda.synchronize()
    apply64_ms = b0.elapsed_time(b1) / 3

    # ---- end to end through the public API (host buffers) -----------------------
    # the same metric: each step copies u from pinned host memory, applies the
    # operator and reads y back
    host_u = u32.cpu().pin_memory()
    host_y = torch.empty_like(host_u).pin_memory()
    du, dy = torch.empty_like(u32), torch.empty_like(u32)
    ne = 10
    torch.cuda.synchronize()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record()
    for _ in range(ne):
        du.copy_(host_u, non_blocking=True)
        mesh.apply_operator(du, dy)
        host_y.copy_(dy, non_blocking=True)
    h1.record()
    torch.cuda.synchronize()
    e2e_apply_ms = h0.elapsed_time(h1) / ne
    # and a whole solve from host data: set_data from host arrays, solve, x to host
    host_x = torch.empty(n_tot, dtype=torch.float64).pin_memory()
    e0 = time.perf_counter()
    mesh.set_data(f=data["f"], a=data["a"], grad_a=data["grad_a"], g=data["g"])
    x.zero_()
    rep_e2e = solve(mesh, x, api.FP32)
    host_x.copy_(x)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - e0
    h2d = data["f"].nbytes + data["a"].nbytes + data["grad_a"].nbytes
    e2e = dict(value=ws * n_tot / (e2e_apply_ms * 1e-3) / 1e9, unit="GDOF/s",
               h2d_bytes_per_step=int(host_u.numel() * 4), d2h_bytes_per_step=int(host_y.numel() * 4),
               solve=dict(tts_s=e2e_s, h2d_bytes=int(h2d), d2h_bytes=int(host_x.numel() * 8),
                          note="set_data from host arrays + mixed solve + x to host"))

    # ---- mixed vs FP64 time-to-solution on a subset of right-hand sides ----------
    cmp = None
    if not args.no_cmp and rank == 0:
        k = min(args.cmp_rhs, args.rhs)
        sub = wl.Problem(pb.mesh, pb.f[:k], pb.g[:k], pb.a, pb.grad_a)
        ms2 = api.Mesh(sub.mesh, n_rhs=k, coef_kind=api.COEF_SCALAR, device=local)
        ms2.set_data(f=data["f"][:k], a=data["a"], grad_a=data["grad_a"])
        if args.precond == "block":
            ms2.setup_block_preconditioner()
        xs = torch.zeros(k * ms2.ndof, dtype=torch.float64, device=dev)
        ms2.pcg_solve(xs, tol=TOL, prec=api.FP64, max_iter=32, raise_on_error=False)  # graph warm-up
        solve(ms2, xs, api.FP32)
        out = {}
        for name, prec in (("mixed", api.FP32), ("fp64", api.FP64)):
            xs.zero_()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record()
            r = ms2.pcg_solve(xs, tol=TOL, prec=prec, inner_tol=args.delta, max_iter=60000,
                              raise_on_error=False, time_limit_s=600)
            c1.record()
            torch.cuda.synchronize()
            out[name] = (c0.elapsed_time(c1) / 1e3, r, xs.clone())
        h = ms2.h1_error(out["mixed"][2], ref=out["fp64"][2])
        h1 = float(np.max(np.sqrt(h[:, 0] / h[:, 1])))
        sols = dict(timed_mixed=x_timed, cmp_mixed=out["mixed"][2].view(k, -1).cpu().numpy(),
                    cmp_fp64=out["fp64"][2].view(k, -1).cpu().numpy())
        cmp = dict(rhs=k, tts_mixed_s=out["mixed"][0], tts_fp64_s=out["fp64"][0],
                   speedup=out["fp64"][0] / out["mixed"][0],
                   iters_mixed=out["mixed"][1]["iterations"], iters_fp64=out["fp64"][1]["iterations"],
                   refreshes=out["mixed"][1]["sweeps"], status_fp64=out["fp64"][1]["status"],
                   rel_res_mixed=out["mixed"][1]["rel_residual"], rel_res_fp64=out["fp64"][1]["rel_residual"],
                   h1_rel_diff_mixed_vs_fp64=h1)
        ms2.close()
        if not args.no_oracle_check:
            cmp["oracle_check"] = oracle_check(args, shard_seed0(rank, args.rhs), k, sols)

    tile_report = None
    if args.precond == "block":
        v, tile, tms = mesh.block_tile(args.W, api.FP32)
        tile_report = dict(variant=v, rows_x_rhs=list(tile),
                           candidates_ms={str(k): round(float(x), 4) for k, x in enumerate(tms) if x > 0})
    if rank == 0:
        cb = cpu_baseline(pb, args.cpu_sample_elems, args.cpu_reps) if ws == 1 else None
        line = dict(
            metric=METRIC, value=value, unit="GDOF/s", n_gpus=ws, steps=args.steps, warmup=args.warmup,
            ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
            data="synthetic",
            config=bench_config(args, mesh.ndof),
            solve=dict(gdof_applies_per_s=solve_rate, iterations=reps[-1]["iterations"], refreshes=reps[-1]["sweeps"],
                       applies=reps[-1]["applies"], rel_residual=reps[-1]["rel_residual"],
                       setup_sample_s=t_sample, setup_set_data_s=t_setdata,
                       setup_block_precond_s=t_prec, precond=args.precond,
                       block_tile=tile_report),
            tts_comparison=cmp,
            apply_ms=dict(fp32=apply_ms, fp64=apply64_ms),
            roofline=dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                          traffic=traffic, traffic_unit="bytes per launch", traffic_source=traffic_src,
                          algorithmic_bytes=int(2 * n_tot * 4),
                          kernel="k_apply<COEF_SCALAR> FP32 (W=8)",
                          note="algorithmic volume flops (3,5,6)-field sum factorisation per (element, rhs); "
                               "peak = FP32 ALU %d SMs x 128 lanes x 2 flops x %.0f MHz (derived: the measured "
                               "peaks hold HBM and bf16 tensor figures only)" % (peaks["sms"], peaks["sm_mhz"])),
            roofline_fp64=dict(bound="alu", achieved=alg_flops / (apply64_ms * 1e-3) / 1e12,
                               peak=peaks["fp64"], unit="TFLOP/s",
                               frac=alg_flops / (apply64_ms * 1e-3) / 1e12 / peaks["fp64"],
                               kernel="k_apply<COEF_SCALAR> FP64 (W=8), the refresh apply of the mixed solve",
                               note="same algorithmic flops; peak = FP64 ALU %d SMs x 2 DFMA/cycle x 2 x %.0f MHz"
                                    % (peaks["sms"], peaks["sm_mhz"])),
            cpu_baseline=cb, e2e=e2e, gpu_launches=int(launches), clocks=clocks,
        )
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
