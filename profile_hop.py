"""Runs the hopping kernel on one workload in one storage form and prints its timing.

A small driver for timing and for ncu captures of a single kernel:

  python profile_hop.py --workload 32^3x64 --form f16:12 --iters 5

It sets up the lattice (gauge copy), packs a Gaussian half field, runs
tm_apply_hopping_eo `iters` times (alternating output parity) and reports the mean
launch time from CUDA events (L2 flushed before each launch unless --warm), the
algorithmic bytes and GB/s.

With --doublet MUBAR,EPSBAR it instead runs `iters` doublet solves (tm_solve_doublet; FP64 for
--form f64:18, reliable-update FP32 sloppy for f32:<links>) on two Gaussian flavour sources and
reports the mean solve time -- a driver for captures of the two-flavour hopping kernel.

With --batch N it runs `iters` batched solves (tm_solve_cg_batch, FP32/FP16 sloppy storage per
--form, delta 1e-3) of N Gaussian sources on the workload's lattice and reports the mean time
-- a driver for captures of the batched hopping kernel.  With --batch N --single the same N
systems are solved one after another with tm_solve_cg (the same form and delta), for comparison.

With --contract it runs `iters` meson contractions (tm_meson_contract) of 12 Gaussian
propagators on the workload's lattice and reports the mean time, bytes and FP64 rate.

With --fma-probe it compiles (nvcc, sm_103a) and runs a probe of the GPU's FMA rates: 8
independent fma.rn.f64 / fma.rn.f32 / packed fma.rn.f32x2 chains per thread, 8 blocks of 256
threads per SM, timed with CUDA events, best of 4 launches.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main():
    import torch

    from paper_0905_3331_gb300 import Lattice, inputs
    from paper_0905_3331_gb300 import build as libbuild

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="32^3x64")
    ap.add_argument("--form", default="f16:12", help="storage:links, storage in f64/f32/f16")
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--warm", action="store_true", help="do not flush L2 between launches")
    ap.add_argument("--parity", type=int, default=-1, help="output parity 0 or 1 (default: alternate)")
    ap.add_argument("--tps", type=int, default=0, help="threads per site 1/2/4 (0: autotuned)")
    ap.add_argument("--doublet", default=None, help="MUBAR,EPSBAR: time doublet solves instead")
    ap.add_argument("--delta", type=float, default=0.001, help="reliable-update delta of the doublet and batched solves")
    ap.add_argument("--contract", action="store_true", help="time meson contractions instead")
    ap.add_argument("--batch", type=int, default=0, help="time batched solves of this many sources")
    ap.add_argument("--single", action="store_true", help="with --batch: solve the sources one at a time")
    ap.add_argument("--fma-probe", action="store_true", help="measure the FP64 / FP32 FMA rates instead")
    args = ap.parse_args()
    if args.fma_probe:
        return fma_probe()
    if args.batch:
        return batch(args)
    if args.doublet:
        return doublet(args)
    if args.contract:
        return contract(args)
    libbuild.build()
    prec = {"f64": 0, "f32": 1, "f16": 2, "df64": 3}[args.form.split(":")[0]]
    nreal = int(args.form.split(":")[1])
    w = inputs.WORKLOADS[args.workload]
    dev = torch.device("cuda:0")
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    if args.tps:
        lat.set_hop_threads(prec, nreal, args.tps)
    lat.set_gauge(w.gauge())
    h = w.V // 2
    nb = lat.half_field_bytes(prec)
    src = inputs.gaussian_spinor(w.T, w.L, w.source_seed, shape_prefix=(args.nrhs,))
    half = np.ascontiguousarray(src.reshape(args.nrhs, -1, 4, 3)[:, :h])
    din = torch.empty(args.nrhs * nb, dtype=torch.uint8, device=dev)
    dout = torch.empty(args.nrhs * nb, dtype=torch.uint8, device=dev)
    lat.pack_half(prec, din, torch.from_numpy(half).to(dev), nrhs=args.nrhs)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    lat.apply_hopping_eo(1, dout, din, prec, nreal, nrhs=args.nrhs)
    torch.cuda.synchronize()
    times = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.iters):
        if not args.warm:
            flush.zero_()
        e0.record(stream)
        lat.apply_hopping_eo(k & 1 if args.parity < 0 else args.parity, dout, din, prec, nreal, nrhs=args.nrhs)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    spinor = {0: 192, 1: 96, 2: 52, 3: 192}[prec]
    elem = {0: 8, 1: 4, 2: 2, 3: 8}[prec]
    per_site = args.nrhs * 2 * spinor + 8 * nreal * elem
    t = statistics.mean(times)
    print(json.dumps({"workload": w.name, "form": args.form, "nrhs": args.nrhs, "h": h,
                      "threads_per_site": lat.hop_threads(prec, nreal),
                      "us": t * 1e6, "bytes_per_site": per_site,
                      "gbs": per_site * h / t / 1e9,
                      "gflops": 1320 * args.nrhs * h / t / 1e9,
                      "l2": "warm" if args.warm else "flushed"}))
    lat.close()


def batch(args):
    import torch

    from paper_0905_3331_gb300 import CG_RELIABLE, Lattice, inputs, solve_cg_batch
    from paper_0905_3331_gb300 import build as libbuild
    libbuild.build()
    prec = {"f32": 1, "f16": 2}[args.form.split(":")[0]]
    nreal = int(args.form.split(":")[1])
    w = inputs.WORKLOADS[args.workload]
    dev = torch.device("cuda:0")
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(w.gauge())
    systems = []
    for k in range(args.batch):
        b = torch.from_numpy(w.source(k)).to(dev)
        systems.append((lat, w.mu, torch.zeros_like(b), b))
    kw = dict(sloppy_prec=prec, sloppy_link=nreal, delta=args.delta)

    def solve():
        if not args.single:
            return solve_cg_batch(systems, **kw)
        out = []
        for _, _, x, b in systems:
            x.zero_()
            out.append(lat.solve_cg(x, b, mode=CG_RELIABLE, **kw))
        return out

    infos = solve()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(args.iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = solve()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.mean(times)
    print(json.dumps({"workload": w.name, "form": args.form, "systems": args.batch,
                      "mode": "single" if args.single else "batched", "ms": t * 1e3,
                      "systems_per_s": args.batch / t, "iters": [i.iters for i in infos],
                      "max_true_rel_residual": max(i.true_rel_residual for i in infos)}))
    lat.close()


def contract(args):
    import torch

    from paper_0905_3331_gb300 import Lattice, inputs
    from paper_0905_3331_gb300 import build as libbuild
    libbuild.build()
    w = inputs.WORKLOADS[args.workload]
    dev = torch.device("cuda:0")
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    props = torch.from_numpy(inputs.gaussian_spinor(w.T, w.L, 7, shape_prefix=(12,))).to(dev)
    out = torch.empty((w.T, 12, 12, 2), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    lat.meson_contract(props, out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(args.iters):
        if not args.warm:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.meson_contract(props, out)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.mean(times)
    nbytes = props.numel() * props.element_size()
    flops = 78 * 12 * 8 * w.V
    print(json.dumps({"workload": w.name, "contract_us": t * 1e6, "bytes": nbytes, "gbs": nbytes / t / 1e9,
                      "fp64_tflops": flops / t / 1e12}))
    lat.close()


def doublet(args):
    import torch

    from paper_0905_3331_gb300 import CG_FP64, CG_RELIABLE, Lattice, inputs
    from paper_0905_3331_gb300 import build as libbuild
    libbuild.build()
    mubar, epsbar = (float(v) for v in args.doublet.split(","))
    prec, nreal = args.form.split(":")
    w = inputs.WORKLOADS[args.workload]
    dev = torch.device("cuda:0")
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(w.gauge())
    b = torch.from_numpy(np.stack([w.source(0), w.source(1)])).to(dev)
    x = torch.zeros_like(b)
    kw = dict(mode=CG_FP64) if prec == "f64" else dict(mode=CG_RELIABLE, sloppy_link=int(nreal), delta=args.delta)
    info = lat.solve_doublet(x, b, mubar, epsbar, **kw)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(args.iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = lat.solve_doublet(x, b, mubar, epsbar, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    print(json.dumps({"workload": w.name, "form": args.form, "doublet": [mubar, epsbar],
                      "ms": statistics.mean(times) * 1e3, "iters": info.iters,
                      "reliable_updates": info.reliable_updates,
                      "true_rel_residual": info.true_rel_residual}))
    lat.close()


FMA_PROBE_SRC = r"""
#include <cstdio>
#include <cuda_runtime.h>
typedef unsigned long long u64;
template <typename T> __device__ __forceinline__ T fma_(T a, T b, T c);
template <> __device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
template <> __device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ float2 fma_(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <typename T> __device__ T seed(int k);
template <> __device__ double seed<double>(int k) { return threadIdx.x * 1e-3 + k; }
template <> __device__ float seed<float>(int k) { return threadIdx.x * 1e-3f + k; }
template <> __device__ float2 seed<float2>(int k) { return make_float2(threadIdx.x * 1e-3f + k, k + 0.5f); }
__device__ double sum_(double v) { return v; }
__device__ double sum_(float v) { return v; }
__device__ double sum_(float2 v) { return v.x + v.y; }
template <typename T> __global__ void k(double* out, T a, T b, int iters) {
  T x[8];
  for (int j = 0; j < 8; ++j) x[j] = seed<T>(j);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma_(x[j], a, b);
  double s = 0; for (int j = 0; j < 8; ++j) s += sum_(x[j]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
template <typename T> double rate(T a, T b, int iters, int lanes, double* out, int blocks) {
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    float ms;
    cudaEventRecord(e0); k<T><<<blocks, 256>>>(out, a, b, iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  return 2.0 * 8 * lanes * iters * (double)blocks * 256 / best / 1e9;
}
int main() {
  int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int blocks = sms * 8;
  double* out; cudaMalloc(&out, sizeof(double) * blocks * 256);
  const double f64 = rate<double>(0.999, 1e-3, 512, 1, out, blocks);
  const double f32 = rate<float>(0.999f, 1e-3f, 4096, 1, out, blocks);
  const double f32x2 = rate<float2>(make_float2(0.999f, 0.999f), make_float2(1e-3f, 1e-3f), 4096, 2, out, blocks);
  printf("{\"fp64_fma_tflops\": %.4f, \"fp32_fma_tflops\": %.3f, \"fp32x2_fma_tflops\": %.3f, \"sms\": %d, \"error\": \"%s\"}\n",
         f64, f32, f32x2, sms, cudaGetErrorString(cudaGetLastError()));
  return 0;
}
"""


def fma_probe():
    import subprocess
    import tempfile
    from paper_0905_3331_gb300 import build as libbuild
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "fma_probe.cu"), os.path.join(d, "fma_probe")
        with open(src, "w") as fh:
            fh.write(FMA_PROBE_SRC)
        subprocess.run([libbuild.nvcc(), *libbuild.ARCH, "-O3", src, "-o", exe], check=True)
        print(subprocess.run([exe], check=True, capture_output=True, text=True).stdout.strip())


if __name__ == "__main__":
    main()
