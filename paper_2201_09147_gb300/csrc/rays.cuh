// Per-ray state machine of one level of multiscale sphere tracing (Alg. 1),
// shared by the SIMT and tensor-core trace kernels.  Each ray slot lives in
// the registers of one thread; slots are refilled from the level's work list
// with warp-aggregated atomics so that tiles stay dense.
#pragma once

#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace sdfnn {

enum : int { kSlotEmpty = 0, kSlotActive = 1, kSlotDone = 2 };

struct Ray {
    int state = kSlotEmpty;
    int idx = 0, nlev = 0, ntot = 0;
    float px = 0.f, py = 0.f, pz = 0.f, vx = 0.f, vy = 0.f, vz = 0.f, tau = 0.f;
};

// Slab test of the ray against [lo, hi]^3: entry distance (>= 0) or -1 on a miss.
// One hardware reciprocal per axis (relative error of a few units in the last
// place: the entry point moves by ~1e-7, far inside every tolerance of the
// trace); a component below the smallest normal float is taken as parallel
// to its slab.
__device__ __forceinline__ float slab_entry(float ox, float oy, float oz, float vx, float vy, float vz, float lo,
                                            float hi) {
    float tn = -INFINITY, tf = INFINITY;
    const float o[3] = {ox, oy, oz}, v[3] = {vx, vy, vz};
    bool miss = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (fabsf(v[c]) >= 0x1p-126f) {
            const float r = __fdividef(1.0f, v[c]);
            const float t1 = (lo - o[c]) * r, t2 = (hi - o[c]) * r;
            tn = fmaxf(tn, fminf(t1, t2));
            tf = fminf(tf, fmaxf(t1, t2));
        } else if (o[c] < lo || o[c] > hi) {
            miss = true;
        }
    }
    tn = fmaxf(tn, 0.0f);
    return (miss || tn > tf) ? -1.0f : tn;
}

__device__ __forceinline__ bool outside_box(float x, float y, float z, float lo, float hi) {
    const float a = lo - kBoxSlack, b = hi + kBoxSlack;
    return x < a || x > b || y < a || y > b || z < a || z > b;
}

// hit >= 0 writes out_hit too (final write of the ray); hit < 0 stores the
// state for the next level only.
__device__ __forceinline__ void write_ray(const LevelArgs& a, int i, float x, float y, float z, float tau, int ntot,
                                          int hit) {
    const int64_t n = a.n;
    a.out_pos[i] = x;
    a.out_pos[n + i] = y;
    a.out_pos[2 * n + i] = z;
    a.out_t[i] = tau;
    if (a.out_iters) a.out_iters[i] = static_cast<uint16_t>(ntot < 65535 ? ntot : 65535);
    if (hit >= 0) a.out_hit[i] = static_cast<uint8_t>(hit);
}

// Fill the slot if it is empty: the slot ends active, or done when the
// level's work list is exhausted.  Rays that miss the box are written out
// on the spot.  Must be called by every lane of the warp.
__device__ __forceinline__ void refill_ray(const LevelArgs& a, Ray& r, long long n_work) {
    bool want = r.state == kSlotEmpty;
    while (__any_sync(0xffffffffu, want)) {
        const long long k = warp_grab(a.grab, want);
        if (!want) continue;
        if (k >= n_work) {
            r.state = kSlotDone;
            want = false;
        } else if (a.in_list == nullptr) {
            const int i = static_cast<int>(k);
            const float ox = a.orig[i], oy = a.orig[a.n + i], oz = a.orig[2 * a.n + i];
            const float vx = a.dir[i], vy = a.dir[a.n + i], vz = a.dir[2 * a.n + i];
            const float tn = slab_entry(ox, oy, oz, vx, vy, vz, a.box_lo, a.box_hi);
            if (tn < 0.0f) {
                write_ray(a, i, ox, oy, oz, 0.0f, 0, 0);
            } else {
                r.idx = i;
                r.px = fmaf(tn, vx, ox);
                r.py = fmaf(tn, vy, oy);
                r.pz = fmaf(tn, vz, oz);
                r.vx = vx;
                r.vy = vy;
                r.vz = vz;
                r.tau = tn;
                r.nlev = 0;
                r.ntot = 0;
                r.state = kSlotActive;
                want = false;
            }
        } else {
            const int i = a.in_list[k];
            r.idx = i;
            r.px = a.out_pos[i];
            r.py = a.out_pos[a.n + i];
            r.pz = a.out_pos[2 * a.n + i];
            r.vx = a.dir[i];
            r.vy = a.dir[a.n + i];
            r.vz = a.dir[2 * a.n + i];
            r.tau = a.out_t[i];
            r.nlev = 0;
            r.ntot = a.out_iters ? a.out_iters[i] : 0;
            r.state = kSlotActive;
            want = false;
        }
    }
}

// One step of Alg. 1 given f(p):  t = f - d;  p += s * t * v;  the level
// ends when t <= eps or the cap is reached; leaving the widened box is a
// miss.  Finished rays are written out, or pushed to the next level's list.
// Must be called by every lane of the warp.
__device__ __forceinline__ void step_ray(const LevelArgs& a, Ray& r, float f) {
    bool push = false;
    if (r.state == kSlotActive) {
        const float t = f - a.d;
        const float step = a.scale * t;
        r.px = fmaf(step, r.vx, r.px);
        r.py = fmaf(step, r.vy, r.py);
        r.pz = fmaf(step, r.vz, r.pz);
        r.tau += step;
        r.nlev += 1;
        r.ntot += 1;
        if (outside_box(r.px, r.py, r.pz, a.box_lo, a.box_hi)) {
            write_ray(a, r.idx, r.px, r.py, r.pz, r.tau, r.ntot, 0);
            r.state = kSlotEmpty;
        } else if (!(t > a.eps) || r.nlev >= a.cap) {
            if (a.is_last) {
                write_ray(a, r.idx, r.px, r.py, r.pz, r.tau, r.ntot, (t <= a.eps) ? 1 : 0);
            } else {
                write_ray(a, r.idx, r.px, r.py, r.pz, r.tau, r.ntot, -1);
                push = true;
            }
            r.state = kSlotEmpty;
        }
    }
    const long long slot = warp_grab(a.out_count, push);
    if (push) a.out_list[slot] = r.idx;
}

// A level with cap 0 passes every ray through unchanged (a miss if it is the
// last level, since it never converged there).  Every lane of the warp.
__device__ __forceinline__ void pass_ray(const LevelArgs& a, Ray& r) {
    bool push = false;
    if (r.state == kSlotActive) {
        write_ray(a, r.idx, r.px, r.py, r.pz, r.tau, r.ntot, a.is_last ? 0 : -1);
        push = !a.is_last;
        r.state = kSlotEmpty;
    }
    const long long slot = warp_grab(a.out_count, push);
    if (push) a.out_list[slot] = r.idx;
}

}  // namespace sdfnn
