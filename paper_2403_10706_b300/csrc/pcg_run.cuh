// The Jacobi PCG of one Gauss-Newton step (Sec. 2.3.1) run by a group of co-resident blocks:
// pcg_run, the body of the persistent PCG kernels and of the persistent GN loop.
#pragma once

#include "grid_sync.cuh"

namespace hysco {

constexpr int kPcgUnroll = 4;

// The PCG of one problem on a group of blocks (the whole grid, or a block range of a batched
// launch): grp.rank is this block's rank in the group, grp.size the group's block count; the
// barriers span the group alone, with the problem's own sync words, whose barrier generation
// `gen` continues from the caller's (the sync words are zeroed once per launch).  RO: grad, d, e
// and 1/diag were written before the launch (read-only path); otherwise by the same launch.
// Returns false when a barrier timed out (the device state then records HYSCO_ETIMEOUT).
template <int P, bool RO = true>
__device__ __forceinline__ bool pcg_run(const Geo& g, const PcgArgs& a, BarrierGroup grp,
                                        float* shf, df32* shd, float4* slots, unsigned& gen) {
  DevState* st = a.st;
  if (st->stop) return true;
  const int T = grp.size * blockDim.x;
  const int gtid = grp.rank * blockDim.x + threadIdx.x;
  const int n4 = g.nfp >> 2;   // float4 groups of the pitched field (padding is zero)
  const int G = a.onchip;
  float4* const rS = slots + threadIdx.x;
  float4* const pS = rS + G * kPcgBlock;
  float4* const hS = pS + G * kPcgBlock;
  float4* const r4 = reinterpret_cast<float4*>(a.r);
  float4* const p4 = reinterpret_cast<float4*>(a.p0);
  float4* const h4 = reinterpret_cast<float4*>(a.Hp);
  auto timed_out = [&]() { if (threadIdx.x == 0) { st->status = -6; st->stop = 1; } };

  float tot[2];
  // ---- init --------------------------------------------------------------------------------
  {
    float arr = 0.f, arz = 0.f;
    for (int i0 = gtid, s0 = 0; i0 < n4; i0 += kPcgUnroll * T, s0 += kPcgUnroll) {
      float4 gv[kPcgUnroll], dv[kPcgUnroll];
#pragma unroll
      for (int u = 0; u < kPcgUnroll; ++u) {
        int i = min(i0 + u * T, n4 - 1);
        gv[u] = ld_in<RO>(reinterpret_cast<const float4*>(a.grad) + i);
        dv[u] = ld_in<RO>(reinterpret_cast<const float4*>(a.invd) + i);
      }
#pragma unroll
      for (int u = 0; u < kPcgUnroll; ++u) {
        int i = i0 + u * T, sl = s0 + u;
        float4 rv = make_float4(a.rhs_sign * gv[u].x, a.rhs_sign * gv[u].y, a.rhs_sign * gv[u].z,
                                a.rhs_sign * gv[u].w);
        float4 zv = make_float4(rv.x * dv[u].x, rv.y * dv[u].y, rv.z * dv[u].z, rv.w * dv[u].w);
        if (i < n4) {
          reinterpret_cast<float4*>(a.x)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (sl < G) rS[sl * kPcgBlock] = rv;
          else r4[i] = rv;
          reinterpret_cast<float4*>(a.z)[i] = zv;
          arr += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
          arz += rv.x * zv.x + rv.y * zv.y + rv.z * zv.z + rv.w * zv.w;
        }
      }
    }
    tot[0] = arr; tot[1] = arz;
  }
  if (!grid_allreduce<2>(tot, a.sync, ++gen, shf, shd, 0, -1, kBarrierSpinCycles, grp)) {
    timed_out();
    return false;
  }
  // scalars in single precision (the sums themselves are double-float accurate)
  const float rr0 = tot[0];
  float rho = tot[1], beta = 0.f, relres = rr0 > 0.f ? 1.f : 0.f;
  bool done = !(rr0 > 0.f);
  int it = 0;
  // x += alpha p.  x is read and written only at the thread's own groups, so no barrier orders
  // it.  On-chip slots: inside the barrier after phase B, between the block's arrival and its
  // wait, where its traffic overlaps the barrier's latency.  Slots in global memory: in phase A
  // of the next iteration, where p is read anyway (x += alpha_{i-1} p_{i-1} before p's update),
  // or by the pass after the loop.  Same operations on every x element either way.
  float al_x = 0.f;   // alpha whose update of the global-memory slots is pending (0: none)
  float4* const x4 = reinterpret_cast<float4*>(a.x);

  for (int i = 0; i < a.max_it && !done; ++i) {
    const bool first = i == 0;
    const float fb = beta;
    // ---- A: w = H z; p = z + beta p; Hp = w + beta Hp ----------------------------------------
    float acc = 0.f;
    for (int t = gtid, sl = 0; t < n4; t += T, ++sl) {
      const bool on = sl < G;
      float4 po = make_float4(0.f, 0.f, 0.f, 0.f), ho = po, pn, hn;
      if (!first) {
        po = on ? pS[sl * kPcgBlock] : p4[t];
        ho = on ? hS[sl * kPcgBlock] : h4[t];
        if (!on) {
          float4 X = i == 1 ? make_float4(0.f, 0.f, 0.f, 0.f) : x4[t];
          X.x = fmaf(al_x, po.x, X.x); X.y = fmaf(al_x, po.y, X.y);
          X.z = fmaf(al_x, po.z, X.z); X.w = fmaf(al_x, po.w, X.w);
          x4[t] = X;
        }
      }
      acc += hv_core<P, true, RO>(g, t, a.z, a.dco, a.eco, fb, first, po, ho, pn, hn);
      if (on) { pS[sl * kPcgBlock] = pn; hS[sl * kPcgBlock] = hn; }
      else { p4[t] = pn; h4[t] = hn; }
    }
    al_x = 0.f;
    float al;
    {
      // only p.Hp crosses blocks here (phase B reads the thread's own groups)
      float t1[1] = {acc};
      if (!grid_allreduce_unordered(t1[0], a.sync, ++gen, shf, shd, 0, -1, kBarrierSpinCycles,
                                    grp)) {
        timed_out();
        return false;
      }
      if (!(t1[0] > 0.f)) { done = true; break; }
      al = rho / t1[0];
      al_x = al;
      // ---- B: r -= alpha Hp, z = r / diag --------------------------------------------------
      float arr = 0.f, arz = 0.f;
      for (int j0 = gtid, s0 = 0; j0 < n4; j0 += kPcgUnroll * T, s0 += kPcgUnroll) {
        float4 hv[kPcgUnroll], dv[kPcgUnroll], rv[kPcgUnroll];
#pragma unroll
        for (int u = 0; u < kPcgUnroll; ++u) {
          // out-of-range slots re-read this thread's own group j0 (never another thread's)
          const bool in = j0 + u * T < n4;
          const int j = in ? j0 + u * T : j0, sl = in ? s0 + u : s0;
          const bool on = sl < G;
          hv[u] = on ? hS[sl * kPcgBlock] : h4[j];
          rv[u] = on ? rS[sl * kPcgBlock] : r4[j];
          dv[u] = ld_in<RO>(reinterpret_cast<const float4*>(a.invd) + j);
        }
#pragma unroll
        for (int u = 0; u < kPcgUnroll; ++u) {
          const int j = j0 + u * T, sl = s0 + u;
          float4 R = rv[u];
          R.x = fmaf(-al, hv[u].x, R.x); R.y = fmaf(-al, hv[u].y, R.y);
          R.z = fmaf(-al, hv[u].z, R.z); R.w = fmaf(-al, hv[u].w, R.w);
          float4 Z = make_float4(R.x * dv[u].x, R.y * dv[u].y, R.z * dv[u].z, R.w * dv[u].w);
          if (j < n4) {
            if (sl < G) rS[sl * kPcgBlock] = R;
            else r4[j] = R;
            reinterpret_cast<float4*>(a.z)[j] = Z;
            arr += R.x * R.x + R.y * R.y + R.z * R.z + R.w * R.w;
            arz += R.x * Z.x + R.y * Z.y + R.z * Z.z + R.w * Z.w;
          }
        }
      }
      tot[0] = arr; tot[1] = arz;
    }
    // on-chip slots: x += alpha p (x = 0 before the first update) while the barrier completes,
    // kPcgUnroll groups' loads in flight at a time so that it fits in the barrier's latency
    auto x_update = [&]() {
      for (int j0 = gtid, s0 = 0; j0 < n4 && s0 < G; j0 += kPcgUnroll * T, s0 += kPcgUnroll) {
        float4 pv[kPcgUnroll], xv[kPcgUnroll];
#pragma unroll
        for (int u = 0; u < kPcgUnroll; ++u) {
          // slots past the range or off chip re-read this thread's own group j0 (slot s0 < G)
          const bool in = j0 + u * T < n4 && s0 + u < G;
          const int j = in ? j0 + u * T : j0, sl = in ? s0 + u : s0;
          pv[u] = pS[sl * kPcgBlock];
          xv[u] = first ? make_float4(0.f, 0.f, 0.f, 0.f) : x4[j];
        }
#pragma unroll
        for (int u = 0; u < kPcgUnroll; ++u) {
          const int j = j0 + u * T;
          float4 X = xv[u];
          X.x = fmaf(al, pv[u].x, X.x); X.y = fmaf(al, pv[u].y, X.y);
          X.z = fmaf(al, pv[u].z, X.z); X.w = fmaf(al, pv[u].w, X.w);
          if (j < n4 && s0 + u < G) x4[j] = X;
        }
      }
    };
    if (!grid_allreduce_then<2>(tot, a.sync, ++gen, shf, shd, x_update, 0, -1,
                                kBarrierSpinCycles, grp)) {
      timed_out();
      return false;
    }
    it = i + 1;
    relres = sqrtf(tot[0]) / sqrtf(rr0);
    if (relres < (float)a.rtol) {
      done = true;
    } else {
      beta = tot[1] / rho;
      rho = tot[1];
    }
  }
  // the last iteration's update of the global-memory slots
  if (al_x != 0.f) {
    for (int t = gtid + G * T, sl = G; t < n4; t += T, ++sl) {
      const float4 pv = p4[t];
      float4 X = it == 1 ? make_float4(0.f, 0.f, 0.f, 0.f) : x4[t];
      X.x = fmaf(al_x, pv.x, X.x); X.y = fmaf(al_x, pv.y, X.y);
      X.z = fmaf(al_x, pv.z, X.z); X.w = fmaf(al_x, pv.w, X.w);
      x4[t] = X;
    }
  }
  if (grp.rank == 0 && threadIdx.x == 0) {
    st->rr0 = rr0;
    st->rho = rho;
    st->beta_cg = beta;
    st->pcg_iter = it;
    st->relres = relres;
    st->pcg_done = 1;
  }
  return true;
}

}  // namespace hysco
