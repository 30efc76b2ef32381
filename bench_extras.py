"""Secondary measurements reported in bench.py's JSON line under "extras".

Each section times one row of the hot path on synthetic, seeded inputs with
CUDA events (kernels) or wall time around a synchronising solve (solvers):

  modes    fp64-unit, fp32 and bf16 operator kernels on the main mesh, and
           the fp32 kernel with G formed from the corner vertices
  sweep    fp64 operator (handle, prepared geometry) and ax_helm on fp64
           geometry at E in {4096, 32768} x lx in {6, 8, 10, 12}; the handle
           at E = 32768 for lx in {3, 4, 5, 7}; lx 14 and 16 at E = 4096
  cg       Poisson solve to a 1e-8 relative residual at E = 32768, lx = 8:
           fp64 Jacobi-CG against fp64 iterative refinement around fp32 and
           bf16-data inner CG
  cg_sweep fp64 Jacobi-CG to 1e-8 at E in {4096, 32768} x lx in {6, 8, 10, 12}
  learned  the same target on the variable-coefficient problem: Jacobi
           flexible CG against the learned element preconditioner in its
           symmetric linear form (trained here by the library's kernels on
           residual/error pairs of 20 plain-CG iterates on an 8^3 mesh: 10,240
           element pairs), in fp64 and inside mixed refinement
  rates    multiply-add throughput per SM and clock (fp64, fp32, packed
           f32x2), the rates that decide the fp64 design (bench_probe.cu,
           built here apart from the library)
  batch    64 meshes, E log-uniform in [64, 8192], lx in {5, 6, 8, 10}: one
           persistent launch (and its CUDA-graph replay) against one launch
           per mesh, fp64 and fp32
  tri_df   prototype of the fp64-accurate on-the-fly trilinear geometry:
           the time to form G per point from the corners in double-float,
           alone (bench_probe.cu), against the HBM time of the 56 bytes of
           stored geometry it would replace
"""
from __future__ import annotations

import os
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))

GKEYS = ("g11", "g22", "g33", "g12", "g13", "g23")


def _events_ms(fn, reps, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _wall(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def _mesh_tensors(ax, synth, n, lx, dev, seed=0):
    import torch
    v = synth.box_vertices(n, seed=seed)
    g = ax.box_geometry(v, lx)
    sh = g["g11"].shape
    t = lambda a: torch.as_tensor(a, device=dev)
    d = {"u": t(synth.uniform(sh, seed=seed + 1)), "h1": t(np.ones(sh))}
    d["dx"], d["dxt"] = (t(a) for a in ax.dmat(lx))
    for k in GKEYS:
        d[k] = t(g[k])
    return d, sh[0]


def sample_elements(nel, count=64):
    """Elements on which the CPU-baseline leg checks every mode against the
    oracle: spread over the mesh, the first and the last included."""
    return np.unique(np.linspace(0, nel - 1, count).round().astype(np.int64))


def mode_outputs(ax, lx, u, h1, dx, dxt, G, corners, xi, wq):
    """Every operator mode of the modes section applied to the same small
    set of elements (fp64 host inputs; G a dict of the six factors): the
    fp64 variants and the operator handle, fp32 and bf16 storage, fp32 with
    G formed from the corners.  Returns {mode: fp64 host output}."""
    import torch
    dev = torch.device("cuda")
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), device=dev).to(dt)
    a64 = [t(u), t(dx), t(dxt), t(h1)] + [t(G[k]) for k in GKEYS]
    out = {}
    w = torch.empty_like(a64[0])
    for name, var in (("f64_native", ax.AX_VARIANT_F64_NATIVE), ("f64_df", ax.AX_VARIANT_F64_DF),
                      ("f64_df_eo", ax.AX_VARIANT_F64_DF_EO)):
        try:
            ax.ax_helm(w, *a64, lx, variant=var)
        except ax.AxError:
            continue
        out[name] = w.cpu().numpy().copy()
    ax.ax_helm(w, *a64, lx)
    out["f64_ax_helm_unprepared"] = w.cpu().numpy().copy()
    op = ax.Operator(lx, a64[1], a64[2], a64[3], *a64[4:])
    op.apply(w, a64[0])
    out["f64_op_prepared"] = w.cpu().numpy().copy()
    for mode, dt, fn in (("f32", torch.float32, ax.ax_helm_f32),
                         ("bf16", torch.bfloat16, ax.ax_helm_bf16)):
        f = [t(u, dt), t(h1, dt)] + [t(G[k], dt) for k in GKEYS]
        w32 = torch.empty(f[0].shape, dtype=torch.float32, device=dev)
        fn(w32, f[0], t(dx, torch.float32), t(dxt, torch.float32), f[1], *f[2:], lx)
        out[mode] = w32.double().cpu().numpy()
    w32 = torch.empty(u.shape, dtype=torch.float32, device=dev)
    ax.ax_helm_trilinear_f32(w32, t(u, torch.float32), t(dx, torch.float32),
                             t(dxt, torch.float32), None, t(corners).reshape(-1), t(xi), t(wq),
                             lx)
    out["f32_trilinear"] = w32.double().cpu().numpy()
    torch.cuda.synchronize()
    return out


def modes(ax, d, lx, nel, hbm_peak):
    import torch
    out = {}
    npts = nel * lx ** 3
    G = [d[k] for k in GKEYS]
    w64 = torch.empty_like(d["u"])
    for name, var in (("f64_native", ax.AX_VARIANT_F64_NATIVE), ("f64_df", ax.AX_VARIANT_F64_DF),
                      ("f64_df_eo", ax.AX_VARIANT_F64_DF_EO)):
        try:
            ms = _events_ms(lambda: ax.ax_helm(w64, d["u"], d["dx"], d["dxt"], d["h1"], *G, lx,
                                               variant=var), 10)
        except ax.AxError:
            continue
        out[name] = {"gdofs": round(npts / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 4),
                     "hbm_frac": round(72.0 * npts / (ms * 1e-3) / 1e9 / hbm_peak, 4)}
    # ax_helm's own choice on the caller's fp64 arrays (no prepared geometry)
    ms = _events_ms(lambda: ax.ax_helm(w64, d["u"], d["dx"], d["dxt"], d["h1"], *G, lx), 10)
    out["f64_ax_helm_unprepared"] = {
        "gdofs": round(npts / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 4),
        "hbm_frac": round(72.0 * npts / (ms * 1e-3) / 1e9 / hbm_peak, 4)}
    op = ax.Operator(lx, d["dx"], d["dxt"], d["h1"], *G)
    if op.info()["prepared"]:
        ms = _events_ms(lambda: op.apply(w64, d["u"]), 10)
        out["f64_op_prepared"] = {"gdofs": round(npts / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 4),
                                  "hbm_frac": round(72.0 * npts / (ms * 1e-3) / 1e9 / hbm_peak, 4)}
    del w64, op
    for mode, dt, bpp in (("f32", torch.float32, 36), ("bf16", torch.bfloat16, 20)):
        f = {k: d[k].to(dt) for k in ("u", "h1") + GKEYS}
        dx32, dxt32 = d["dx"].float(), d["dxt"].float()
        w = torch.empty(f["u"].shape, dtype=torch.float32, device=d["u"].device)
        fn = ax.ax_helm_f32 if mode == "f32" else ax.ax_helm_bf16
        ms = _events_ms(lambda: fn(w, f["u"], dx32, dxt32, f["h1"], *[f[k] for k in GKEYS], lx),
                        30)
        out[mode] = {"gdofs": round(npts / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 4),
                     "hbm_frac": round(bpp * npts / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                     "bytes_per_point": bpp}
        del f, w
    # fp32 with G formed from the corner vertices (h1 = 1): u and w only.
    # Two buffer sets alternate (2 x 134 MB > L2) so no launch reads the
    # previous one's data from L2.
    from paper_2506_20994_gb300 import synth
    n = round(nel ** (1.0 / 3.0))
    if n ** 3 == nel:
        dev = d["u"].device
        xi, wq = (torch.as_tensor(a, device=dev) for a in ax.gll(lx))
        cor = torch.as_tensor(ax.box_corners(synth.box_vertices(n, seed=0)), device=dev)
        dx32, dxt32 = d["dx"].float(), d["dxt"].float()
        us = [d["u"].float(), d["u"].float().clone()]
        ws = [torch.empty_like(us[0]) for _ in range(2)]
        k = [0]

        def tri():
            i = k[0] & 1
            k[0] += 1
            ax.ax_helm_trilinear_f32(ws[i], us[i], dx32, dxt32, None, cor.reshape(-1), xi, wq,
                                     lx)
        ms = _events_ms(tri, 30)
        bpp = 8.0 + 192.0 / lx ** 3
        out["f32_trilinear"] = {"gdofs": round(npts / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 4),
                                "hbm_frac": round(bpp * npts / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                                "bytes_per_point": round(bpp, 3), "h1": "constant 1",
                                "l2": "two alternating buffer sets (268 MB)"}
        del us, ws, cor
    return out


def sweep(ax, synth, dev, hbm_peak):
    import torch
    out = {}
    for n in (16, 32):
        for lx in (6, 8, 10, 12):
            d, nel = _mesh_tensors(ax, synth, n, lx, dev)
            w = torch.empty_like(d["u"])
            G = [d[k] for k in GKEYS]
            op = ax.Operator(lx, d["dx"], d["dxt"], d["h1"], *G)
            ms = _events_ms(lambda: op.apply(w, d["u"]), 10)
            ms_raw = _events_ms(lambda: ax.ax_helm(w, d["u"], d["dx"], d["dxt"], d["h1"], *G, lx),
                                10)
            npts = nel * lx ** 3
            out[f"E{nel}_lx{lx}"] = {"gdofs": round(npts / (ms * 1e-3) / 1e9, 2),
                                     "ms": round(ms, 4),
                                     "hbm_frac": round(72.0 * npts / (ms * 1e-3) / 1e9 / hbm_peak,
                                                       4),
                                     "gdofs_paper_convention": round(
                                         nel * (lx - 1) ** 3 / (ms * 1e-3) / 1e9, 2),
                                     "raw_geometry_ms": round(ms_raw, 4)}
            del d, w, op
    # the paper's lower orders (lx 3-7): the operator handle at E = 32768; it
    # prepares geometry for even lx >= 6 and applies ax_helm's choice otherwise
    for lx in (3, 4, 5, 7):
        d, nel = _mesh_tensors(ax, synth, 32, lx, dev)
        w = torch.empty_like(d["u"])
        G = [d[k] for k in GKEYS]
        op = ax.Operator(lx, d["dx"], d["dxt"], d["h1"], *G)
        ms = _events_ms(lambda: op.apply(w, d["u"]), 10)
        npts = nel * lx ** 3
        out[f"E{nel}_lx{lx}"] = {"gdofs": round(npts / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 4),
                                 "hbm_frac": round(72.0 * npts / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                                 "gdofs_paper_convention": round(
                                     nel * (lx - 1) ** 3 / (ms * 1e-3) / 1e9, 2),
                                 "prepared": bool(op.info()["prepared"])}
        del d, w, op
    # high order: the double-float k-loop kernel (ax_helm's choice) against the
    # fp64 units, E = 4096
    for lx in (14, 16):
        d, nel = _mesh_tensors(ax, synth, 16, lx, dev)
        w = torch.empty_like(d["u"])
        G = [d[k] for k in GKEYS]
        args = (w, d["u"], d["dx"], d["dxt"], d["h1"], *G, lx)
        ms = _events_ms(lambda: ax.ax_helm(*args), 5)
        ms_native = _events_ms(lambda: ax.ax_helm(*args, variant=ax.AX_VARIANT_F64_NATIVE), 5)
        npts = nel * lx ** 3
        out[f"E{nel}_lx{lx}"] = {"gdofs": round(npts / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 4),
                                 "hbm_frac": round(72.0 * npts / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                                 "kernel": "double-float k-loop",
                                 "fp64_units_ms": round(ms_native, 4)}
        del d, w
    return out


def cg(ax, synth, oracle_f, dev):
    v = synth.box_vertices(32, seed=0)
    P = ax.Poisson(v, 8, device=dev)
    P.set_check_every(8)
    b = P.rhs(oracle_f)
    out = {"workload": "Poisson, f = 3 pi^2 sin sin sin, Dirichlet, E=32768, lx=8, tol 1e-8"}
    t, (x, its, rel, rc) = _wall(lambda: P.cg(b, tol=1e-8))
    out["f64_jacobi_cg"] = {"s": round(t, 4), "iters": its, "relres": rel, "status": rc}
    for name, mode, itol in (("f32_ir", ax.AX_PREC_F32, 1e-4), ("bf16_ir", ax.AX_PREC_BF16, 1e-2)):
        t2, (x2, no, ni, rel2, rc2) = _wall(lambda: P.mpcg(b, mode=mode, tol=1e-8,
                                                           inner_tol=itol))
        t2b, (x2, no, ni, rel2, rc2) = _wall(lambda: P.mpcg(b, mode=mode, tol=1e-8,
                                                            inner_tol=itol))
        out[name] = {"s": round(t2b, 4), "first_call_s": round(t2, 4), "outer": no,
                     "inner_iters": ni, "relres": rel2, "status": rc2,
                     "speedup_vs_f64_cg": round(t / t2b, 3)}
    return out


def cg_sweep(ax, synth, oracle_f, dev):
    """Jacobi-PCG to 1e-8 on the sweep meshes (E in {4096, 32768} x lx in
    {6, 8, 10, 12}), fp64."""
    out = {}
    for n in (16, 32):
        for lx in (6, 8, 10, 12):
            P = ax.Poisson(synth.box_vertices(n, seed=0), lx, device=dev)
            P.set_check_every(8)
            b = P.rhs(oracle_f)
            P.cg(b, tol=1e-8, maxit=3)  # warm-up
            t, (x, its, rel, rc) = _wall(lambda: P.cg(b, tol=1e-8))
            out[f"E{n ** 3}_lx{lx}"] = {"s": round(t, 4), "iters": its, "relres": rel,
                                        "status": rc,
                                        "ms_per_iter": round(t / max(its, 1) * 1e3, 4)}
            del P, b, x
    return out


def learned(ax, synth, oracle_f, dev):
    lx = 8
    coef = ax.fourier_coefficient(1)
    out = {"workload": "Poisson, variable h1 in [0.5, 2] (8 Fourier modes), E=32768, lx=8, "
                       "tol 1e-8"}
    # train on residual/error pairs of plain CG on an 8^3 mesh (element-local
    # network: it transfers to the larger mesh)
    # 8^3 elements x 20 CG iterates = 10,240 element residual/error pairs
    Ps = ax.Poisson(synth.box_vertices(8, seed=0), lx, h1=coef, device=dev)
    bs = Ps.rhs(oracle_f)
    iterates = (1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 112, 128)
    n_hid = 48
    M = ax.Mlp(lx ** 3, n_hid, arch=ax.AX_MLP_SYM,
               params=ax.mlp_init_params(lx ** 3, n_hid, seed=1, arch=ax.AX_MLP_SYM))
    t_pairs, (R, E) = _wall(lambda: ax.iterate_pairs(Ps, bs, iterates=iterates))
    t_train, loss = _wall(lambda: ax.train_energy(Ps, M, R, E, epochs=100, lr=2e-3))
    out["training"] = {"arch": "symmetric linear, n_hid 48", "iterates": int(R.shape[0]),
                       "element_pairs": int(R.shape[0]) * Ps.nelv,
                       "params": lx ** 3 * n_hid,
                       "params_note": "free parameters of the tied form (one lx^3 x 48 basis "
                                      "W used as W and W^T); %d stored in the flat layout"
                                      % M.nparams,
                       "pair_s": round(t_pairs, 3), "train_s": round(t_train, 3),
                       "final_rel_energy_err": loss}
    t_setup = t_pairs + t_train
    del Ps, R, E
    P = ax.Poisson(synth.box_vertices(32, seed=0), lx, h1=coef, device=dev)
    P.set_check_every(8)
    b = P.rhs(oracle_f)
    P.cg(b, tol=1e-8, maxit=3)  # warm-up
    # the baseline: plain fp64 Jacobi-preconditioned CG on the same problem
    tc, (x, ic, rc_, sc) = _wall(lambda: P.cg(b, tol=1e-8))
    out["f64_jacobi_cg"] = {"s": round(tc, 4), "iters": ic, "relres": rc_, "status": sc}

    def vs_cg(t):
        return {"speedup_vs_f64_jacobi_cg": round(tc / t, 3),
                "speedup_vs_f64_jacobi_cg_with_training": round(tc / (t + t_setup), 3)}
    t0, (x, i0, r0, f0, s0) = _wall(lambda: P.fcg(b, None, tol=1e-8))
    out["f64_jacobi_fcg"] = {"s": round(t0, 4), "iters": i0, "status": s0}
    t1, (x, i1, r1, f1, s1) = _wall(lambda: P.fcg(b, M, tol=1e-8))
    out["f64_learned_fcg"] = {"s": round(t1, 4), "iters": i1, "fallbacks": f1, "status": s1,
                              **vs_cg(t1)}
    P.mpfcg(b, None, tol=1e-8)  # converts the fp32 operator data once
    t2, (x, no, ni, r2, f2, s2) = _wall(lambda: P.mpfcg(b, None, tol=1e-8, inner_tol=1e-4))
    out["f32_ir_jacobi"] = {"s": round(t2, 4), "outer": no, "inner_iters": ni, "status": s2,
                            "speedup_vs_f64_jacobi": round(t0 / t2, 3)}
    t3, (x, no, ni, r3, f3, s3) = _wall(lambda: P.mpfcg(b, M, tol=1e-8, inner_tol=1e-4))
    out["f32_ir_learned"] = {"s": round(t3, 4), "outer": no, "inner_iters": ni,
                             "fallbacks": f3, "status": s3,
                             "speedup_vs_f64_jacobi": round(t0 / t3, 3), **vs_cg(t3)}
    out["f32_ir_jacobi"].update(vs_cg(t2))
    out["training_s"] = round(t_setup, 3)
    return out


def batch(ax, synth, dev, hbm_peak):
    import torch
    specs = synth.batch_meshes(seed=0)
    out = {"meshes": len(specs), "elements": int(sum(a * b * c for a, b, c, _ in specs)),
           "lx_set": sorted({s[3] for s in specs})}
    for dtype, name, tdt, bpp in ((ax.AX_BATCH_F64, "f64", torch.float64, 72),
                                  (ax.AX_BATCH_F32, "f32", torch.float32, 36)):
        meshes = []
        for q, (nx, ny, nz, lx) in enumerate(specs):
            v = synth.box_vertices(nx, ny, nz, seed=q)
            g = ax.box_geometry(v, lx)
            sh = g["g11"].shape
            t = lambda a: torch.as_tensor(a, device=dev, dtype=tdt)
            m = {"lx": lx, "u": t(synth.uniform(sh, seed=100 + q)), "h1": t(np.ones(sh))}
            m["dx"], m["dxt"] = (t(a) for a in ax.dmat(lx))
            for k in GKEYS:
                m[k] = t(g[k])
            m["w"] = torch.empty_like(m["u"])
            meshes.append(m)
        B = ax.Batch(meshes, dtype=dtype)
        info = B.info()
        ms_p = _events_ms(lambda: B.launch(), 10)
        ms_g = _events_ms(lambda: B.launch(graph=True), 10)

        def separate():
            for m in meshes:
                args = (m["w"], m["u"], m["dx"], m["dxt"], m["h1"], *[m[k] for k in GKEYS],
                        m["lx"])
                (ax.ax_helm if dtype == ax.AX_BATCH_F64 else ax.ax_helm_f32)(*args)
        ms_s = _events_ms(separate, 5)
        pts = sum(m["u"].numel() for m in meshes)
        out[name] = {"persistent_ms": round(ms_p, 4), "graph_ms": round(ms_g, 4),
                     "separate_launches_ms": round(ms_s, 4),
                     "gdofs_graph": round(pts / (ms_g * 1e-3) / 1e9, 2),
                     "hbm_frac_graph": round(bpp * pts / (ms_g * 1e-3) / 1e9 / hbm_peak, 4),
                     "items": info["items"], "blocks": info["blocks"], "graph_launches": 1,
                     "kernels_in_graph": 1}
        del B, meshes
    return out


def _probe_lib():
    """bench_probe.cu, built here with nvcc into _build/ and loaded on its own
    (it is not part of the library)."""
    import ctypes
    import shutil
    import subprocess
    src = os.path.join(ROOT, "bench_probe.cu")
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libaxprobe.so")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = so + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                        "-gencode", "arch=compute_103a,code=sm_103a", "-I", ROOT,
                        "-I", os.path.join(ROOT, "include"), src, "-o", tmp], check=True)
        os.replace(tmp, so)
    return ctypes.CDLL(so)


def tri_df_probe(ax, synth, dev, n=32, lx=8):
    """The fp64-accurate on-the-fly trilinear geometry prototype (bench_probe.cu):
    time to compute G per point from the corners in double-float at E = n^3,
    and its element-0 G against ax_box_geometry's fp64 G."""
    import ctypes
    import numpy as np
    import torch
    lib = _probe_lib()
    v = synth.box_vertices(n, seed=0)
    cor = torch.as_tensor(ax.box_corners(v), device=dev).reshape(-1).contiguous()
    xi, wq = (torch.as_tensor(a, device=dev) for a in ax.gll(lx))
    g0 = torch.zeros(6 * lx ** 3, dtype=torch.float64, device=dev)
    ms = ctypes.c_float()
    rc = lib.bench_probe_tri_df(ctypes.c_void_p(cor.data_ptr()), ctypes.c_void_p(xi.data_ptr()),
                                ctypes.c_void_p(wq.data_ptr()), ctypes.c_int(n ** 3),
                                ctypes.c_int(20), ctypes.c_void_p(g0.data_ptr()),
                                ctypes.byref(ms),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise RuntimeError(f"bench_probe_tri_df failed: {rc}")
    geo = ax.box_geometry(v[:2, :2, :2], lx)  # element 0 of the same mesh
    ref = np.stack([geo[k][0].reshape(-1) for k in ("g11", "g22", "g33", "g12", "g13", "g23")])
    got = g0.cpu().numpy().reshape(6, -1)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    npts = n ** 3 * lx ** 3
    return {"what": "G from the 8 corners per point in double-float (k-loop schedule), alone",
            "E": n ** 3, "lx": lx, "ms": round(ms.value, 4),
            "ns_per_point_all_sms": round(ms.value * 1e6 / npts, 4),
            "rel_err_g_element0_vs_fp64": err,
            "stored_geometry_bytes_saved_per_point": 56,
            "hbm_time_of_those_bytes_ms": round(56 * npts / 6785.9e9 * 1e3, 4)}


def probe_rates() -> dict:
    """Multiply-add throughput per SM and clock of the current device (fp64,
    fp32, packed f32x2): bench_probe.cu, built here with nvcc into _build/
    and loaded on its own (it is not part of the library)."""
    import ctypes
    import torch
    lib = _probe_lib()
    rates = (ctypes.c_double * 3)()
    rc = lib.bench_probe_rates(rates, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise RuntimeError(f"bench_probe_rates failed: {rc}")
    return {"fp64_fma": rates[0], "fp32_fma": rates[1], "fp32x2_fma": rates[2]}


def rates(ax):
    """Multiply-add throughput per SM and clock (fp64, fp32, packed f32x2)
    and what the fp64 one implies for an fp64-unit operator at lx = 8."""
    import torch
    r = probe_rates()
    props = torch.cuda.get_device_properties(0)
    r["sms"] = props.multi_processor_count
    # Listing 2's flops per fp64 byte at lx = 8: (12 lx^4 + 18 lx^3) / (72 lx^3)
    intensity = (12 * 8 ** 4 + 18 * 8 ** 3) / (72 * 8 ** 3)
    r["fp64_ratio_to_fp32"] = round(r["fp64_fma"] / r["fp32_fma"], 4)
    r["lx8_fp64_flop_per_byte"] = round(intensity, 3)
    return r


def run_extras(ax, host, d, lx, nel, stream, hbm_peak, which):
    from paper_2506_20994_gb300 import synth
    dev = d["u"].device
    out = {}
    sections = {
        "modes": lambda: modes(ax, d, lx, nel, hbm_peak),
        "sweep": lambda: sweep(ax, synth, dev, hbm_peak),
        "cg": lambda: cg(ax, synth, synth.poisson_source, dev),
        "cg_sweep": lambda: cg_sweep(ax, synth, synth.poisson_source, dev),
        "learned": lambda: learned(ax, synth, synth.poisson_source, dev),
        "batch": lambda: batch(ax, synth, dev, hbm_peak),
        "rates": lambda: rates(ax),
        "tri_df": lambda: tri_df_probe(ax, synth, dev),
    }
    for name, fn in sections.items():
        if name not in which:
            continue
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as exc:  # report, do not lose the main line
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
        out[name + "_wall_s"] = round(time.perf_counter() - t0, 2)
    return out
