#!/usr/bin/env python
"""Benchmark: spacetime DOF-updates/s of the MTP-SAT evolution on one GB300.

Workload (default): 3D Maxwell, unit cube graded toward (0,0,0) with size ratio 8,
32^3 x 6 = 196608 tets, p = 4 (q = 5 stages, m = 8 sub-intervals), eps = 4 in the
ball of radius 0.25 around the centre, mu = 1, Gaussian E pulse (width 0.05, seeded
centre), PEC walls, T = 0.5, tents pitched with causality factor 0.5.

One step = one full evolve 0 -> T through every tent (all layers), state resident
in HBM.  metric value = sum_i N_dof,i m q / step time (Sec. 5.2 of the paper).
Also reported: the same metric end to end through the host-buffer C-ABI call, the
plain FP64 GPU path on a truncated window of layers (same window for both modes),
the roofline of the tent kernel, and the oracle on the host cores.

--impl reference runs the FP64 CPU oracle (the only reference implementation of
this method here) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import hashlib  # noqa: E402

import numpy as np  # noqa: E402

FP32_SM_LANES = 128            # FP32 FMA lanes per SM (Blackwell)
KERNEL_SOURCES = ["paper_1906_11029_gb300/csrc/mtp_kernels.cuh", "paper_1906_11029_gb300/csrc/mtp_launch.cuh"]
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per tent of the tent kernels on the
# graded 32^3 workload, from an ncu capture of a window of layers (scaled per tent), keyed by
# (precision, kernel) and stamped with the hash of the kernel sources at capture time: a
# stamp that no longer matches the sources means the kernel changed since, and the bench
# reports traffic null.
TRAFFIC_BYTES_PER_TENT = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum on the launch that applies layers
    # 1000..1099 (81 105 tents) of the graded 32^3 p = 4 workload: 1.145 GB + 0.757 GB
    ("fp32", "tent_persistent_kernel"): {"bytes_per_tent": 23455.2, "sources": "215962c12a1e8c1c"},
}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_tent(precision, kernel):
    rec = TRAFFIC_BYTES_PER_TENT.get((precision, kernel))
    if rec is None or rec["sources"] != kernel_source_hash():
        return None
    return rec["bytes_per_tent"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def make_workload(name):
    import mtp_synth as S
    if name == "graded":
        return S.graded_sphere(32, 4, 0.5)
    if name == "cube":
        return S.cube_mode(16, 3, 1.0)
    if name == "small":
        return S.graded_sphere(8, 4, 0.1)
    raise SystemExit(f"unknown workload {name}")


def initial_lattice(w):
    import mtp_synth as S
    pts = S.lattice_points(w.verts, w.elems, w.p)
    E, H = w.init(pts, 0.0)
    fs = [0, 1, 5] if w.dim == 2 else [0, 1, 2, 3, 4, 5]
    u = np.concatenate([E, H], -1)[..., fs]
    mat = np.where(np.array(fs) < 3, 1.0, 0.0)
    scale = mat[None, None, :] * w.eps[:, None, None] + (1 - mat[None, None, :]) * w.mu[:, None, None]
    return np.ascontiguousarray(u * scale)


def flops_per_dof_update(dim, p):
    """Algorithmic minimum per DOF-update: volume d nf Np^2 + facets d nf 2 Nfp Np + mass solve and
    M' 2 nf^2 Np multiply-adds per element and operator application, x2 flops, / (nf Np)."""
    nf = 3 if dim == 2 else 6
    nb = (p + 1) * (p + 2) // 2 if dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6
    nfb = p + 1 if dim == 2 else (p + 1) * (p + 2) // 2
    mac = dim * nf * nb * nb + dim * nf * 2 * nfb * nb + 2 * nf * nf * nb
    return 2.0 * mac / (nf * nb)


def window_dofs(w, tents, lb, le, p, nrhs=1):
    nf = 3 if w.dim == 2 else 6
    nb = (p + 1) * (p + 2) // 2 if w.dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6
    psize = np.bincount(w.elems.ravel(), minlength=len(w.verts))
    lp = tents["layer_ptr"]
    v = tents["vertex"][lp[lb]:lp[le]]
    return float(psize[v].sum()) * nf * nb * (2 * p) * (p + 1) * nrhs


class Clocks:
    """nvidia-smi sampler (every 200 ms) started before and stopped after the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows)}


def cpu_baseline_sample(workload, n_tents, seed=7, procs=1, warmup=0, steps=1):
    """Time the FP64 oracle (test infrastructure, as it stands) on a bounded sample of the
    workload: the first n_tents tents (in layer order, from the flat front t = 0) applied to a
    seeded random state, `warmup` untimed and `steps` timed repetitions.  With procs > 1 the
    tents of each layer (independent, Sec. 2) are spread over a pool of that many processes.
    Runs in a child process with one BLAS thread per process; returns the JSON it prints."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", workload,
                        "--cpu-tents", str(n_tents), "--seed", str(seed), "--cpu-rounds", "80",
                        "--cpu-procs", str(procs), "--warmup", str(warmup), "--steps", str(steps)],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_ORACLE = {}


def _oracle_init(workload, barrier):
    from oracle.mesh import Mesh as OMesh
    from oracle.mtp import Discretization
    w = make_workload(workload)
    _ORACLE["disc"] = Discretization(OMesh(w.verts, w.elems, w.eps, w.mu), w.p)
    barrier.wait()


def _oracle_tent(job):
    V, dt, tau, Yp = job
    return _ORACLE["disc"].sat_tent(V, dt, tau, Yp)


def cpu_worker(args):
    from oracle.mesh import Mesh as OMesh
    from oracle.mtp import Discretization
    from oracle.pitch import pitch_tents
    w = make_workload(args.cpu_worker)
    disc = Discretization(OMesh(w.verts, w.elems, w.eps, w.mu), w.p)
    tents = pitch_tents(w.verts, w.elems, w.eps, w.mu, w.T, w.causality, max_rounds=args.cpu_rounds)
    n = min(args.cpu_tents, len(tents["vertex"]))
    layers = tents["layer"][:n]
    pool = None
    if args.cpu_procs > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(args.cpu_procs)
        pool = ctx.Pool(args.cpu_procs, initializer=_oracle_init, initargs=(args.cpu_worker, barrier))
        pool.map(abs, range(args.cpu_procs))          # every worker has built its oracle
    rates, secs = [], []
    for rep in range(args.warmup + args.steps):
        rng = np.random.default_rng(args.seed + rep)
        Y = rng.standard_normal((len(w.elems), disc.nf * disc.nb))
        tau = np.zeros(len(w.verts))
        dofs = 0.0
        t0 = time.perf_counter()
        t = 0
        while t < n:                          # (layer, vertex) order: any prefix respects the DAG
            e = t
            while e < n and layers[e] == layers[t]:
                e += 1
            jobs = []
            for i in range(t, e):
                V = int(tents["vertex"][i])
                jobs.append((V, float(tents["t_top"][i]) - float(tents["t_bot"][i]), tau, Y[disc.mesh.patch[V]]))
            res = pool.map(_oracle_tent, jobs) if pool else [disc.sat_tent(*j) for j in jobs]
            for i, (slots, Yp) in zip(range(t, e), res):
                V = int(tents["vertex"][i])
                Y[slots] = Yp
                tau[V] = float(tents["t_top"][i])
                dofs += len(disc.mesh.patch[V]) * disc.nf * disc.nb * (2 * w.p) * (w.p + 1)
            t = e
        dt = time.perf_counter() - t0
        if rep >= args.warmup:
            rates.append(dofs / dt)
            secs.append(dt)
    if pool:
        pool.close()
        pool.join()
    print(json.dumps({"value": float(np.mean(rates)), "values": rates, "seconds": float(np.mean(secs)),
                      "tents": n, "procs": args.cpu_procs}))


def run_reference(args):
    """The FP64 CPU oracle on all host cores (the tents of a layer spread over a process pool),
    bounded sample per step (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(args.workload)
    cores = min(host_cores(), args.cpu_max_procs)
    n = args.ref_tents * cores
    r = cpu_baseline_sample(args.workload, n, seed=100, procs=cores, warmup=args.warmup, steps=args.steps)
    if "error" in r:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + r["error"][-200:]}))
        return
    rate, secs = r["value"], r["seconds"]
    sample = f"first {r['tents']} tents (layer order) per step, seeded random state, FP64 numpy oracle"
    line = {
        "impl": "reference", "metric": "spacetime DOF-updates/s", "value": rate,
        "unit": "DOF-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "elems": int(len(w.elems)), "p": w.p, "sample": sample},
        "cpu_baseline": {"value": rate, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample + f", tents of each layer over {cores} processes"},
        "e2e": {"value": rate, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_profile(args):
    """Profiling driver: build the workload, then apply layers [a, b) once (no timing)."""
    import torch
    import paper_1906_11029_gb300 as mtp
    a, b = (int(x) for x in args.profile_window.split(":"))
    w = make_workload(args.workload)
    prec = mtp.MTP_FP32 if args.precision == "fp32" else mtp.MTP_FP64
    flags = mtp.MTP_FLAG_LAYER_LAUNCHES if args.layer_launches else 0
    mesh = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=prec, flags=flags)
    tents = mesh.pitch(w.T, w.causality)
    tents.set_variant(args.variant)
    state = mesh.state_from_lattice(torch.tensor(initial_lattice(w)[None], device="cuda"))
    if a > 0:
        tents.evolve_layers(state, 0, a)
    tents.evolve_layers(state, a, b)
    torch.cuda.synchronize()
    launches = int(np.count_nonzero(np.diff(tents.get()["layer_ptr"][a:b + 1]))) if args.layer_launches else 1
    print(json.dumps({"profile_window": [a, b], "launches": launches, "workload": w.name,
                      "kernel": "tent_layer_kernel" if args.layer_launches else "tent_persistent_kernel"}))


def run_profile_evolve(args):
    """Profiling driver: build the workload and run one full evolve (the persistent kernel)."""
    import torch
    import paper_1906_11029_gb300 as mtp
    w = make_workload(args.workload)
    prec = mtp.MTP_FP32 if args.precision == "fp32" else mtp.MTP_FP64
    mesh = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=prec)
    tents = mesh.pitch(w.T, w.causality)
    state = mesh.state_from_lattice(torch.tensor(initial_lattice(w)[None], device="cuda"))
    tents.evolve(state)
    torch.cuda.synchronize()
    print(json.dumps({"profile_evolve": w.name, "tents": tents.info["n_tents"]}))


def run_many(args):
    """Many-instance workload: 64 independent PEC cube problems, n ~ U{6..20}, p ~ U{2,3,4}
    (seed 4), 4 Gaussian-pulse right-hand sides each, FP32, T = 0.5, one persistent launch."""
    import torch
    import mtp_synth as S
    import paper_1906_11029_gb300 as mtp
    recipe = S.many_instances(args.many_count, seed=4, n_rhs=4)
    insts = []
    t0 = time.perf_counter()
    for r in recipe:
        v, e = S.cube_mesh(r["n"])
        one = np.ones(len(e))
        m = mtp.Mesh(3, v, e, one, one, p=r["p"], precision=mtp.MTP_FP32, n_rhs=4)
        t = m.pitch(r["T"], 0.5)
        pts = S.lattice_points(v, e, r["p"])
        vals = np.stack([np.concatenate(S.gaussian_pulse(c, r["width"])(pts), -1) for c in r["centres"]])
        st = m.state_from_lattice(torch.tensor(np.ascontiguousarray(vals), device="cuda"))
        del vals, pts
        insts.append((m, t, st))
    batch = mtp.Batch([t for _, t, _ in insts])
    setup_s = time.perf_counter() - t0
    dofs = batch.info["spacetime_dofs"]
    for _ in range(args.warmup):
        batch.evolve([st.clone() for _, _, st in insts])
    torch.cuda.synchronize()
    work = [st.clone() for _, _, st in insts]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for _ in range(args.steps):
        for wk, (_, _, st) in zip(work, insts):
            wk.copy_(st)
        a.record()
        batch.evolve(work)
        b.record()
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
    print(json.dumps({"metric": "spacetime DOF-updates/s", "value": args.steps * dofs / (ms / 1e3),
                      "unit": "DOF-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms / args.steps, "higher_is_better": True, "dtype": "f32",
                      "data": "synthetic", "gpu_launches": args.steps,
                      "config": {"workload": f"many_instances_{args.many_count}x4rhs",
                                 "tents": batch.info["n_tents"], "dof_updates_per_step": dofs,
                                 "elems_total": int(sum(m.info["n_elems"] for m, _, _ in insts)),
                                 "setup_s": setup_s}}))


def lattice_interpolation(dim, p_from, p_to):
    """Matrix taking values of a degree-p_from polynomial at its lattice points to its values at
    the degree-p_to lattice points of the same simplex (exact; monomials in the reference
    coordinates of the sorted-vertex lattice)."""
    import itertools
    import mtp_synth as S
    exps = [e for e in itertools.product(range(p_from + 1), repeat=dim) if sum(e) <= p_from]

    def vander(p):
        pts = S.lattice_multi_indices(dim, p).astype(float) / p
        return np.array([[np.prod(pt ** np.array(e)) for e in exps] for pt in pts])
    return vander(p_to) @ np.linalg.inv(vander(p_from))


def run_equal_error(args):
    """Discretisation error of the p = 4 graded workload estimated against p = 5 on the same mesh
    and tents (u4 interpolated exactly to the p = 5 lattice), next to the distance of each
    FP32-state mode (and of kernel variant 3, the volume term on tcgen05) from the FP32 SIMT path
    and from each other."""
    import torch
    import mtp_synth as S
    import paper_1906_11029_gb300 as mtp
    w4 = make_workload(args.workload)
    out, times, dofs = {}, {}, {}
    TC5 = "tc5"   # MTP_FP32 with kernel variant 3
    runs = [(5, mtp.MTP_FP32), (4, mtp.MTP_FP32), (4, mtp.MTP_TF32), (4, mtp.MTP_TF32X3), (4, mtp.MTP_FP32_SPLIT)]
    if w4.dim == 3 and w4.p == 4:
        runs.append((4, TC5))
    if args.equal_error_fp64:
        runs.append((4, mtp.MTP_FP64))
    for p, prec in runs:
        w = S.graded_sphere(32, p, 0.5) if args.workload == "graded" else w4
        mesh = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=p, precision=mtp.MTP_FP32 if prec == TC5 else prec)
        tents = mesh.pitch(w.T, w.causality)
        if prec == TC5:
            tents.set_variant(3)
        st = mesh.state_from_lattice(torch.tensor(initial_lattice(w)[None], device="cuda"))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        tents.evolve(st)
        b.record()
        torch.cuda.synchronize()
        times[(p, prec)] = a.elapsed_time(b)
        dofs[(p, prec)] = tents.info["spacetime_dofs"]
        out[(p, prec)] = mesh.state_to_lattice(st).cpu().numpy()[0]
        del mesh, tents, st
    I = lattice_interpolation(3, 4, 5)
    u5 = out[(5, mtp.MTP_FP32)]
    up = lambda u4: np.einsum("kl,elf->ekf", I, u4)
    ref = out[(4, mtp.MTP_FP32)]
    rel = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))
    names = {mtp.MTP_FP32: "fp32", mtp.MTP_TF32: "tf32", mtp.MTP_TF32X3: "tf32x3", mtp.MTP_FP64: "fp64",
             mtp.MTP_FP32_SPLIT: "fp32split", TC5: "tcgen05_variant3"}
    res = {"workload": w4.name, "e_disc_p4_vs_p5": rel(up(ref), u5),
           "ms": {f"p{p}_{names[q]}": v for (p, q), v in times.items()}}
    for q in (mtp.MTP_TF32, mtp.MTP_TF32X3, mtp.MTP_FP32_SPLIT, TC5):
        if (4, q) in out:
            res[f"{names[q]}_vs_fp32"] = rel(out[(4, q)], ref)
    if (4, mtp.MTP_FP64) in out:
        # the whole evolve to T in FP64: each FP32-state mode against it, and against e_disc
        u64 = out[(4, mtp.MTP_FP64)]
        res["e_disc_fp64_p4_vs_p5"] = rel(up(u64), u5)
        for q in (mtp.MTP_FP32, mtp.MTP_TF32, mtp.MTP_TF32X3, mtp.MTP_FP32_SPLIT, TC5):
            if (4, q) not in out:
                continue
            d = rel(out[(4, q)], u64)
            res[f"{names[q]}_vs_fp64_full_T"] = d
            res[f"{names[q]}_vs_fp64_over_e_disc"] = d / res["e_disc_fp64_p4_vs_p5"]
        rate = lambda k: dofs[k] / (times[k] / 1e3)
        res["fp64_value"] = rate((4, mtp.MTP_FP64))
        res["fp32_value"] = rate((4, mtp.MTP_FP32))
        res["fp32split_value"] = rate((4, mtp.MTP_FP32_SPLIT))
        res["fp32_speedup_vs_fp64_full_T"] = times[(4, mtp.MTP_FP64)] / times[(4, mtp.MTP_FP32)]
    print(json.dumps(res))


def adjoint_timing(reps=3):
    """The adjoint workload (8^3 x 6 tets, p = 2, eps ~ U[1, 3] seeded, T = 0.5, FP64, tents
    pitched for wave speed 1): milliseconds of one forward evolve and of one mtp_adjoint (forward
    pass with checkpoints, recomputation with the compact patch tape, reverse sweep), best of
    `reps` after a warm-up."""
    import torch
    import mtp_synth as S
    import paper_1906_11029_gb300 as mtp
    w = S.adjoint_cube(8, 2, 0.5)
    m = mtp.Mesh(3, w.verts, w.elems, w.eps, w.mu, p=w.p)
    t = m.pitch(w.T, 0.5, wavespeed=np.ones(len(w.elems)))
    st0 = m.state_from_lattice(torch.tensor(initial_lattice(w)[None], device="cuda"))
    lamT = torch.randn_like(st0)
    lam0 = torch.empty_like(st0)
    ge = torch.empty(len(w.elems), dtype=torch.float64, device="cuda")
    gm = torch.empty_like(ge)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fw, ad = [], []
    for r in range(reps + 1):
        x = st0.clone()
        a.record(); t.evolve(x); b.record(); torch.cuda.synchronize()
        fw.append(a.elapsed_time(b))
        a.record(); mtp.mtp_adjoint(t.h, st0, lamT, lam0, ge, gm); b.record(); torch.cuda.synchronize()
        ad.append(a.elapsed_time(b))
    f, g = min(fw[1:]), min(ad[1:])
    return {"workload": w.name, "layers": t.info["n_layers"], "tents": t.info["n_tents"], "forward_ms": f,
            "adjoint_ms": g, "adjoint_over_forward": g / f}


def run_rk4_study(args):
    """2D TE cavity (Sec. 5.1 convergence study, FP64): lattice l2 errors of SAT and of the
    Y-substituted classical RK4 tent stepper (MTP_FLAG_SUBSTITUTED_RK4) on the same tents, and
    their distance (the RK4 time-stepping error), for p = 1..4 and n = 4..64."""
    import torch
    import mtp_synth as S
    import paper_1906_11029_gb300 as mtp
    rows = []
    for p in (1, 2, 3, 4):
        for n in (4, 8, 16, 32, 64):
            w = S.te_square(n, p, 0.25)
            pts = S.lattice_points(w.verts, w.elems, p)
            E0, H0 = w.exact(pts, 0.0)
            ET, HT = w.exact(pts, w.T)
            v0 = np.ascontiguousarray(np.concatenate([E0, H0], -1)[..., [0, 1, 5]])
            ex = np.concatenate([ET, HT], -1)[..., [0, 1, 5]]
            out = {}
            for flags in (0, mtp.MTP_FLAG_SUBSTITUTED_RK4):
                m = mtp.Mesh(2, w.verts, w.elems, w.eps, w.mu, p=p, precision=mtp.MTP_FP64, flags=flags)
                t = m.pitch(w.T, w.causality)
                st = m.state_from_lattice(torch.tensor(v0[None], device="cuda"))
                t.evolve(st)
                out[flags] = m.state_to_lattice(st).cpu().numpy()[0]
            rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
            rows.append({"p": p, "n": n, "sat": rel(out[0], ex), "rk4": rel(out[mtp.MTP_FLAG_SUBSTITUTED_RK4], ex),
                         "rk4_minus_sat": rel(out[mtp.MTP_FLAG_SUBSTITUTED_RK4], out[0])})
            print(json.dumps(rows[-1]), flush=True)


def run_autotune(args):
    """Run the autotuner (paper_1906_11029_gb300/tune.py) on the workload's own initial data with a
    fresh cache and print its record: every (precision, kernel shape variant) candidate with the
    milliseconds of each launch configuration on the timed window of layers."""
    import paper_1906_11029_gb300.tune as tune
    w = make_workload(args.workload)
    cache = os.path.join(tempfile.mkdtemp(), "tune.json")
    prec, launch, rec = tune.autotune(w.dim, w.verts, w.elems, w.eps, w.mu, w.p, w.T, initial_lattice(w)[None],
                                      accuracy="fp32", causality_factor=w.causality, cache=cache)
    print(json.dumps({"workload": w.name, "choice": {"precision": prec, "variant": rec["variant"], "launch": launch,
                                                     "launch_name": rec["launch_name"]},
                      "candidates": rec["candidates"]}))


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank gets it); `dist` None for one process."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, dofs_per_step, max_ms):
    """Units of all ranks (each rank evolves its own replica) over the slowest rank's time."""
    return world * steps * dofs_per_step / (max_ms / 1e3)


def run_mtp(args):
    import torch
    import paper_1906_11029_gb300 as mtp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    peaks, peak_kind = load_peaks()
    w = make_workload(args.workload)
    prec = mtp.MTP_FP32 if args.precision == "fp32" else mtp.MTP_FP64
    t0 = time.perf_counter()
    flags = mtp.MTP_FLAG_LAYER_LAUNCHES if args.layer_launches else 0
    mesh = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=prec, flags=flags)
    t1 = time.perf_counter()
    tents = mesh.pitch(w.T, w.causality)
    if args.variant:
        tents.set_variant(args.variant)
    if args.launch:
        tents.set_launch(args.launch)
    t2 = time.perf_counter()
    tents_dev = mesh.pitch(w.T, w.causality, device=True)    # same tent list, rounds on the GPU
    t3 = time.perf_counter()
    del tents_dev
    tl = tents.get()
    n_layers = tents.info["n_layers"]
    persistent = not args.layer_launches
    launches_per_step = 1 if persistent else int(np.count_nonzero(np.diff(tl["layer_ptr"])))
    dofs = tents.info["spacetime_dofs"]
    vals0 = torch.tensor(initial_lattice(w)[None], device="cuda")
    state0 = mesh.state_from_lattice(vals0)
    del vals0
    work = state0.clone()
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        work.copy_(state0)
        tents.evolve(work)
    torch.cuda.synchronize()
    probe = mtp.mtp_probe_rates()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        work.copy_(state0)
        ev[k][0].record(stream)
        tents.evolve(work)
        ev[k][1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    total_ms = start.elapsed_time(end)
    kern_ms = sum(a.elapsed_time(b) for a, b in ev)
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    value = whole_job_rate(world, args.steps, dofs, total_ms)

    # roofline of the tent kernel (the evolve is the tent-kernel graph); denominators: the FMA
    # rates measured on this device by mtp_probe_rates (before the timed region), next to the
    # unit-count figure from the device's SM count and maximum clock
    fl = flops_per_dof_update(w.dim, w.p)
    launch_ms = kern_ms / (args.steps * launches_per_step)
    flops_per_launch = dofs * fl / launches_per_step
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    unit_peak = n_sms * FP32_SM_LANES * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    if prec == mtp.MTP_FP32:
        peak, src = probe["fp32_fma"], "mtp_probe_rates FP32 FMA loop on this device, this run"
    else:
        peak, src = probe["fp64_fma"], "mtp_probe_rates FP64 FMA loop on this device, this run"
    achieved = flops_per_launch / (launch_ms / 1e3) / 1e12
    kname = "tent_persistent_kernel" if persistent else "tent_layer_kernel"
    # the stored traffic is the default kernel's (variant 0, occupancy-limit DAG walk)
    default_kernel = args.variant == 0 and args.launch == 0
    tpl = traffic_per_tent(args.precision, kname) if args.workload == "graded" and default_kernel else None
    traffic = None if tpl is None else tpl * tents.info["n_tents"] / launches_per_step
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": f"{kname}<{args.precision},3,{w.p}>", "kernel_variant": args.variant, "launch": args.launch, "peak_source": src,
                "probe_tflops": probe, "fp32_unit_count_peak": unit_peak, "sms": n_sms,
                "frac_of_unit_count_peak": achieved / unit_peak if prec == mtp.MTP_FP32 else None,
                "kernel_sources": kernel_source_hash()}

    # end to end through the host-buffer entry point (pinned buffers, copies in the timed region)
    h_in = state0.cpu().pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    tents.evolve_host(h_in, h_out)
    torch.cuda.synchronize()
    e2e_steps = 1
    barrier()
    te0 = time.perf_counter()
    for _ in range(e2e_steps):
        tents.evolve_host(h_in, h_out)
    te1 = time.perf_counter()
    nbytes = h_in.numel() * h_in.element_size()
    e2e = {"value": world * e2e_steps * dofs / (te1 - te0), "unit": "DOF-updates/s",
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
           "call": "mtp_evolve_host (pinned host buffers)"}

    # plain FP64 GPU path vs this path on the same truncated window of layers
    fp64 = None
    if args.fp64_window > 0 and prec != mtp.MTP_FP64:
        lw = max(1, int(args.fp64_window * n_layers))
        wd = window_dofs(w, tl, 0, lw, w.p)
        mesh64 = mtp.Mesh(w.dim, w.verts, w.elems, w.eps, w.mu, p=w.p, precision=mtp.MTP_FP64)
        tents64 = mesh64.pitch(w.T, w.causality)
        s64 = mesh64.state_from_lattice(torch.tensor(initial_lattice(w)[None], device="cuda"))
        s64w = s64.clone()
        tents64.evolve_layers(s64w, 0, 1)
        torch.cuda.synchronize()
        s64w.copy_(s64)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        tents64.evolve_layers(s64w, 0, lw)
        b.record(stream)
        torch.cuda.synchronize()
        ms64 = a.elapsed_time(b)
        work.copy_(state0)
        a.record(stream)
        tents.evolve_layers(work, 0, lw)
        b.record(stream)
        torch.cuda.synchronize()
        ms32 = a.elapsed_time(b)
        u64 = mesh64.state_to_lattice(s64w).cpu().numpy()
        u32 = mesh.state_to_lattice(work).cpu().numpy()
        fp64 = {"window_layers": lw, "window_dof_updates": wd, "fp64_value": wd / (ms64 / 1e3),
                "this_path_value_same_window": wd / (ms32 / 1e3), "speedup_vs_fp64": ms64 / ms32,
                "rel_l2_vs_fp64_on_window": float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64))}
        del mesh64, tents64, s64, s64w

    adj = adjoint_timing() if rank == 0 and not args.no_adjoint else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = min(host_cores(), args.cpu_max_procs)
        r = cpu_baseline_sample(args.workload, args.cpu_tents * cores, procs=cores)
        r1 = cpu_baseline_sample(args.workload, args.cpu_tents)
        cpu = {"value": r.get("value"), "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
               "sample": f"first {r.get('tents')} tents (layer order) of the same workload, seeded random "
                         f"state, FP64 numpy oracle, tents of each layer over {cores} processes, "
                         f"{r.get('seconds', 0):.1f} s",
               "one_core": {"value": r1.get("value"), "sample": f"first {r1.get('tents')} tents, "
                                                                 f"{r1.get('seconds', 0):.1f} s"},
               **({"error": (r.get("error") or "") + (r1.get("error") or "")} if "error" in r or "error" in r1 else {})}

    if rank == 0:
        line = {
            "metric": "spacetime DOF-updates/s", "value": value, "unit": "DOF-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == mtp.MTP_FP32 else "f64", "data": "synthetic",
            "config": {"workload": w.name, "elems": int(len(w.elems)), "p": w.p, "q": w.p + 1, "m": 2 * w.p,
                       "T": w.T, "tents": tents.info["n_tents"], "layers": n_layers,
                       "dof_updates_per_step": dofs, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "state larger than L2 (%.0f MB)" % (state0.numel() * state0.element_size() / 1e6),
                       "pitch_s": t2 - t1, "pitch_device_s": t3 - t2, "mesh_s": t1 - t0},
            "clocks": clk, "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, "fp64_gpu": fp64, "adjoint": adj,
            "peaks": peak_kind,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mtp", choices=["mtp", "reference"])
    ap.add_argument("--workload", default="graded", choices=["graded", "cube", "small", "many"])
    ap.add_argument("--many-count", type=int, default=64)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--fp64-window", type=float, default=0.02)
    ap.add_argument("--layer-launches", action="store_true", help="one launch per layer instead of the DAG walk")
    ap.add_argument("--variant", type=int, default=0, help="tent kernel shape variant (mtp_tents_set_variant)")
    ap.add_argument("--launch", type=int, default=0, choices=[0, 1],
                    help="DAG walk at the occupancy limit (0) or with one CTA per SM (1) (mtp_tents_set_launch)")
    ap.add_argument("--cpu-tents", type=int, default=80, help="oracle baseline: tents (per process)")
    ap.add_argument("--cpu-rounds", type=int, default=80)
    ap.add_argument("--ref-tents", type=int, default=20, help="reference arm: tents per host core per step")
    ap.add_argument("--cpu-procs", type=int, default=1, help="oracle worker: processes over the tents of a layer")
    ap.add_argument("--cpu-max-procs", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing extra")
    ap.add_argument("--cpu-worker", default=None)
    ap.add_argument("--profile-window", default=None, help="a:b -> apply layers [a, b) once and exit")
    ap.add_argument("--profile-evolve", action="store_true", help="run one full evolve and exit")
    ap.add_argument("--equal-error", action="store_true", help="p=4 precision modes against p=5")
    ap.add_argument("--equal-error-fp64", action="store_true",
                    help="with --equal-error: also one full FP64 p=4 evolve (about 10 min on the graded workload)")
    ap.add_argument("--rk4-study", action="store_true", help="SAT vs substituted RK4 convergence table (2D, FP64)")
    ap.add_argument("--autotune", action="store_true", help="run the autotuner on the workload and print its record")
    ap.add_argument("--seed", type=int, default=7)
    args = ap.parse_args()
    if args.cpu_worker:
        return cpu_worker(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_window:
        return run_profile(args)
    if args.profile_evolve:
        return run_profile_evolve(args)
    if args.workload == "many":
        return run_many(args)
    if args.equal_error:
        return run_equal_error(args)
    if args.rk4_study:
        return run_rk4_study(args)
    if args.autotune:
        return run_autotune(args)
    return run_mtp(args)


if __name__ == "__main__":
    main()
