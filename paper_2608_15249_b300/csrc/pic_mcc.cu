// pic_mcc.cu -- null-collision Monte Carlo of the electrons against a uniform
// neutral background (the G_collision module of Sec. 2.2, which implements the
// null-collision method), with constant cross sections: isotropic elastic
// scattering with the recoil loss 2 m/M (1 - cos chi), and excitation above a
// threshold energy (the electron loses the threshold, then scatters isotropically).
//
// The method bounds the total collision frequency by nu' = n_g (sig_el + sig_exc)
// vmax, makes a fraction P = 1 - exp(-nu' dt) of the particles candidates, and lets a
// candidate of speed v undergo process j with probability nu_j(v) / nu', the rest
// being null collisions.  Random numbers come from a counter-based generator keyed
// by (seed, step, particle id, draw), so a particle's draws do not depend on where
// the sort has put it: the output function of SplitMix64 (Steele, Lea and Flood,
// 2014) applied to seed + (counter + 1) * 0x9E3779B97F4A7C15 with counter =
// step * 2^34 + id * 4 + draw; a draw is the top 24 bits.  The candidate test is an
// integer compare against round(P 2^24).
//
// One streaming pass: each particle's id is read and drawn once; the few candidates
// are compacted per warp before their velocities are read and rewritten; collision
// counts are summed per warp and added to three device counters.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pic_internal.cuh"

namespace apk {

namespace {

constexpr int MCC_THREADS = 256;

__device__ __forceinline__ uint32_t draw24(uint64_t seed, uint64_t step, uint32_t id, int k)
{
    const uint64_t ctr = (step << 34) | ((uint64_t)id << 2) | (uint64_t)k;
    uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)(z >> 40);
}

// The collision of one candidate (draws 1..3), in place; returns the process
// (0 elastic, 1 excitation, -1 null) and flags a candidate above the bound.
__device__ __forceinline__ int collide_one(ParticlesF32 p, int64_t i, uint32_t id,
                                           const MccParams &c, uint64_t step, bool *over)
{
    const float inv24 = 1.0f / 16777216.0f;
    float *vp[3] = {p.v + i, p.v + p.stride + i, p.v + 2 * p.stride + i};
    const float v[3] = {*vp[0], *vp[1], *vp[2]};
    const float v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const float speed = sqrtf(v2);
    const float energy = c.half_m * v2;
    const float nu_el = c.ng_sig_el * speed;
    const float nu_exc = energy >= c.eps_exc ? c.ng_sig_exc * speed : 0.0f;
    *over = nu_el + nu_exc > c.nu_max;
    const float u1 = (float)draw24(c.seed, step, id, 1) * inv24;
    // cos chi = 1 - 2 u2, u2 = (r2 + 1/2) / 2^24.  With t the smaller of u2 and 1 - u2
    // (both (k + 1/2) / 2^24 with k < 2^23, exact in FP32), cos chi = +-(1 - 2 t) and
    // sin chi = 2 sqrt(t (1 - t)): near-forward and near-backward scattering keep
    // their small sin chi, which 1 - cos^2 chi in FP32 would round away.
    const uint32_t r2 = draw24(c.seed, step, id, 2);
    const bool fwd = r2 < (1u << 23);
    const float t2 = ((float)(fwd ? r2 : 16777215u - r2) + 0.5f) * inv24;
    const float cchi = fwd ? 1.0f - 2.0f * t2 : 2.0f * t2 - 1.0f;
    float snew;
    int kind;
    if (u1 < nu_el / c.nu_max) {
        snew = speed * sqrtf(1.0f - c.two_mass_ratio * (1.0f - cchi));
        kind = 0;
    } else if (u1 < (nu_el + nu_exc) / c.nu_max) {
        snew = sqrtf(fmaxf(v2 - c.two_eps_over_m, 0.0f));
        kind = 1;
    } else {
        return -1;  // null collision
    }
    // new direction: vhat cos chi + sin chi (e1 cos phi + e2 sin phi), with the
    // orthonormal basis (e1, e2) perpendicular to vhat of Duff et al. (2017)
    const float u3 = (float)draw24(c.seed, step, id, 3) * inv24;
    float sp, cp;
    sincospif(2.0f * u3, &sp, &cp);
    const float schi = 2.0f * sqrtf(t2 * (1.0f - t2));
    float n[3] = {1.0f, 0.0f, 0.0f};
    if (speed > 0.0f) {
        const float is = 1.0f / speed;
        n[0] = v[0] * is;
        n[1] = v[1] * is;
        n[2] = v[2] * is;
    }
    const float sgn = n[2] >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sgn + n[2]);
    const float b = n[0] * n[1] * a;
    const float e1[3] = {1.0f + sgn * n[0] * n[0] * a, sgn * b, -sgn * n[0]};
    const float e2[3] = {b, sgn + n[1] * n[1] * a, -n[1]};
#pragma unroll
    for (int k = 0; k < 3; ++k) *vp[k] = snew * (n[k] * cchi + schi * (e1[k] * cp + e2[k] * sp));
    return kind;
}

// Each warp takes chunks of MCC_CHUNK particles: every lane reads its share of the
// ids as four 16-byte loads issued together (lane l holds ids 128 r + 4 l + k), draws
// for each, and the candidates are packed into a per-warp list with a ballot and a
// population count; the list is then processed 32 at a time, so the long collision
// path runs with full lanes instead of once per warp that happens to hold a
// candidate.  (The order of the list does not matter: each candidate's collision
// depends only on its own id and velocity.)  The last, partial chunk reads its ids
// one by one.
constexpr int MCC_CHUNK = 512;

__global__ void __launch_bounds__(MCC_THREADS)
    k_mcc(ParticlesF32 p, MccParams c, uint64_t step, unsigned long long *__restrict__ counts)
{
    __shared__ uint32_t s_list[MCC_THREADS / 32][MCC_CHUNK];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *list = s_list[wib];
    int n_el = 0, n_exc = 0, n_over = 0;
    const int64_t nchunks = (p.np + MCC_CHUNK - 1) / MCC_CHUNK;
    const int64_t gwarp = ((int64_t)blockIdx.x * MCC_THREADS + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * MCC_THREADS) >> 5;
    for (int64_t ch = gwarp; ch < nchunks; ch += nwarps) {
        const int64_t base = ch * MCC_CHUNK;
        uint32_t ids[MCC_CHUNK / 32];
        const bool full = base + MCC_CHUNK <= p.np;
        if (full) {
            const uint4 *src = reinterpret_cast<const uint4 *>(p.id + base);
#pragma unroll
            for (int r = 0; r < MCC_CHUNK / 128; ++r) {
                const uint4 q = __ldg(src + r * 32 + lane);
                ids[4 * r] = q.x;
                ids[4 * r + 1] = q.y;
                ids[4 * r + 2] = q.z;
                ids[4 * r + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < MCC_CHUNK / 32; ++k) {
                const int64_t i = base + (k >> 2) * 128 + lane * 4 + (k & 3);
                ids[k] = i < p.np ? p.id[i] : 0u;
            }
        }
        int m = 0;  // candidates listed so far (warp-uniform)
#pragma unroll
        for (int k = 0; k < MCC_CHUNK / 32; ++k) {
            const int j = (k >> 2) * 128 + lane * 4 + (k & 3);
            const bool cand = (full || base + j < p.np) && draw24(c.seed, step, ids[k], 0) < c.thr;
            const unsigned ball = __ballot_sync(0xffffffffu, cand);
            if (cand) list[m + __popc(ball & ((1u << lane) - 1u))] = (uint32_t)j;
            m += __popc(ball);
        }
        __syncwarp();
        for (int q = lane; q < m; q += 32) {
            const int64_t i = base + list[q];
            bool over = false;
            const int kind = collide_one(p, i, p.id[i], c, step, &over);
            n_el += kind == 0;
            n_exc += kind == 1;
            n_over += over;
        }
        __syncwarp();  // the list is rewritten by the next chunk
    }
    n_el = __reduce_add_sync(0xffffffffu, n_el);
    n_exc = __reduce_add_sync(0xffffffffu, n_exc);
    n_over = __reduce_add_sync(0xffffffffu, n_over);
    if (lane == 0) {
        if (n_el) atomicAdd(counts + 0, (unsigned long long)n_el);
        if (n_exc) atomicAdd(counts + 1, (unsigned long long)n_exc);
        if (n_over) atomicAdd(counts + 2, (unsigned long long)n_over);
    }
}

__global__ void __launch_bounds__(MCC_THREADS) k_iota(uint32_t *__restrict__ id, int64_t np)
{
    for (int64_t i = (int64_t)blockIdx.x * MCC_THREADS + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * MCC_THREADS)
        id[i] = (uint32_t)i;
}

int mcc_blocks(int64_t np)
{
    const int sms = sm_count();
    const int64_t need = (np + (int64_t)MCC_CHUNK * (MCC_THREADS / 32) - 1) /
                         ((int64_t)MCC_CHUNK * (MCC_THREADS / 32));
    const int64_t cap = (int64_t)sms * 8;
    const int64_t b = need < cap ? need : cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

MccParams make_mcc_params(double density, double sigma_el, double sigma_exc, double eps_exc,
                          double mass_ratio, double vmax, double m, double dt, uint64_t seed)
{
    MccParams c{};
    const double nu_max = density * (sigma_el + sigma_exc) * vmax;
    const double P = 1.0 - exp(-nu_max * dt);
    c.seed = seed;
    c.thr = (uint32_t)floor(P * 16777216.0 + 0.5);
    c.ng_sig_el = (float)(density * sigma_el);
    c.ng_sig_exc = (float)(density * sigma_exc);
    c.nu_max = (float)nu_max;
    c.eps_exc = (float)eps_exc;
    c.two_eps_over_m = (float)(2.0 * eps_exc / m);
    c.two_mass_ratio = (float)(2.0 * mass_ratio);
    c.half_m = (float)(0.5 * m);
    return c;
}

cudaError_t launch_mcc(ParticlesF32 p, const MccParams &c, uint64_t step,
                       unsigned long long *counts, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), st);
    if (e != cudaSuccess || p.np == 0 || c.thr == 0) return e;
    k_mcc<<<mcc_blocks(p.np), MCC_THREADS, 0, st>>>(p, c, step, counts);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_iota(uint32_t *id, int64_t np, cudaStream_t st)
{
    if (np == 0) return cudaSuccess;
    k_iota<<<mcc_blocks(np), MCC_THREADS, 0, st>>>(id, np);
    note_launch();
    return cudaGetLastError();
}

}  // namespace apk
