// Fused row passes of the FP32 stepper: one kernel per row pass instead of
// an inverse and a forward pass through memory.
//
// The six-kernel step (stepper_impl.cuh) writes the physical fields of each
// row pass to memory and reads them back in the next one, because the
// finite differences across rows (D_y omega in the advection term, D_y du in
// the penalisation curl) need neighbouring rows.  Here a block walks down a
// strip of R rows two at a time (one packed complex transform per row pair)
// and keeps the inverse transforms of three consecutive row pairs of the
// array that is differenced across rows in a ring in shared memory (pairs
// t-1, t, t+1 around pair t), so each row pass reads only x-spectra and
// writes only an x-spectrum:
//
//   k_row_roll<RHS_*>  X1 (omega, ring), X2, X3 (u', v)  -> X4 = x-spectrum of N
//   k_row_roll<PEN_*>  X2 (u*, ring), X1 (omega*), X3 (v*) -> X1 = x-spectrum of
//                      omega^{n+1}, and W (= omega^{n+1}) on the last step of a run
//
// With the column passes (k_col_poisson; k_col_update reading N from X4) a
// step is four kernels and moves about a third fewer bytes, but it performs
// about 10% more transforms (the halo pairs, and omega transformed again
// instead of read): where the transforms, not the memory traffic, bound the
// step, it is not faster.  The arithmetic per point is that of row_value: the
// same centred differences of the same values, with omega taken from the
// inverse transform of its x-spectrum (scaled by 1/nx, a power of two).
//
// Pipelining: blocks are persistent and run a list of steps (per strip, one
// step loading the first two ring pairs, then one step per row pair).  The
// x-spectra of step i+1 are copied global -> shared by cp.async while step i
// transforms; the per-row operands of the pointwise stage (base-derived
// fields, penalisation coefficients) are issued one step ahead as a second
// copy group.  Every wait is a cp.async.wait_group, which completes with the
// copies themselves.
//
// Shape: G = 2048/nx strips side by side (G nx = 2048 row points per pair
// step), 512 threads: the three inverse transforms of a step (the ring pair
// and two more sequences) for all G strips at 8 elements a thread (two
// rounds; the FP32 radix-8 pass with compensated twiddles needs about 100
// registers, which 512 threads leave room for), the forward transform also
// at 8 (fewer passes and one twiddle table for both directions).
// Shared memory 40 G (nx + nx/16) + 56 G nx bytes (197 KB).
#pragma once

namespace nsstab {

constexpr int kRollThreads = 512;
constexpr int kRollPoints = 2048;   // G * nx

// Shared memory of a fused row pass over G strips of nx points (pts = G nx):
// five padded sequences, the staged x-spectra and the per-row operands.
inline size_t roll_smem(int pts) { return (size_t)40 * padded_len(pts, 2) + (size_t)56 * pts; }

struct RollShape {
    int R;           // rows per strip (even, divides ny)
    int G;           // strips per unit, transformed side by side
    int upm;         // units per member: ny / (R G)
    int nunits;      // members * upm
    int write_w;     // PEN: also store omega^{n+1} to W
    int do_fft;      // PEN: forward transform omega^{n+1} into X1
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Offsets of member m's arrays: its own fields and spectra, and the
// per-parameter-set arrays of its set (as in member_view).
struct RollOff {
    size_t fo, co, so;
};
__device__ __forceinline__ RollOff roll_off(const Fields<float>& f, int m) {
    const int set = m / f.bper;
    return {(size_t)m * f.fs, (size_t)m * f.cs, (size_t)set * f.fs};
}

// Position in a block's list of steps: unit (member, G strips) and step s
// (0: first two ring pairs; s >= 1: ring pair s and row pair t = s - 1).
struct RollPos {
    int unit, s;
};

__device__ __forceinline__ bool roll_active(const Fields<float>& f, const RollShape& rs, int unit) {
    return !f.active || f.active[unit / rs.upm];
}

__device__ __forceinline__ RollPos roll_first(const Fields<float>& f, const RollShape& rs) {
    int u = blockIdx.x;
    while (u < rs.nunits && !roll_active(f, rs, u)) u += gridDim.x;
    return {u, 0};
}

__device__ __forceinline__ RollPos roll_next(const Fields<float>& f, const RollShape& rs, RollPos p) {
    if (p.s < rs.R / 2) return {p.unit, p.s + 1};
    int u = p.unit + gridDim.x;
    while (u < rs.nunits && !roll_active(f, rs, u)) u += gridDim.x;
    return {u, 0};
}

template <int MODE> struct RollArrays {
    static constexpr bool PEN = (MODE == FWD_PEN_NL || MODE == FWD_PEN_LIN);
    static constexpr bool AUX = (MODE != FWD_RHS_NL);   // per-row operands staged one step ahead
};

// Copy the x-spectra of step p into the staging area: per strip three
// arrays of nx/2 16-byte row pairs [g][3][nx/2].  s = 0: the ring array's
// pairs -1 and 0; s >= 1: its pair s, then the two arrays of row pair s - 1.
template <int MODE>
__device__ __forceinline__ void roll_issue_spectra(const Fields<float>& f0, const RollShape& rs, RollPos p,
                                                   float4* stage) {
    if (p.unit >= rs.nunits) return;
    constexpr bool PEN = RollArrays<MODE>::PEN;
    const int m = p.unit / rs.upm, grp = p.unit % rs.upm;
    const RollOff o = roll_off(f0, m);
    const int nh = f0.nxh, ny = f0.ny;
    const float2* ring = (PEN ? f0.X2 : f0.X1) + o.co;
    const float2* ma = (PEN ? f0.X1 : f0.X2) + o.co;
    const float2* mb = f0.X3 + o.co;
    const int lognh = f0.logx - 1;
#pragma unroll 1
    for (int e = threadIdx.x; e < rs.G * nh; e += blockDim.x) {
        const int k = e & (nh - 1), g = e >> lognh;
        const int j0 = (grp * rs.G + g) * rs.R;
        float4* dst = stage + (size_t)g * 3 * nh + k;
        const size_t col = (size_t)k * ny;
        if (p.s == 0) {
            cp_async16(dst, ring + col + ((j0 - 2 + ny) & (ny - 1)));
            cp_async16(dst + nh, ring + col + j0);
        } else {
            const int a = j0 + 2 * (p.s - 1);
            cp_async16(dst, ring + col + ((j0 + 2 * p.s) & (ny - 1)));
            cp_async16(dst + nh, ma + col + a);
            cp_async16(dst + 2 * nh, mb + col + a);
        }
    }
}

// Per-row operands of row pair t = p.s - 1 of every strip, [g][8][nx]:
// RHS_LIN: U_b, V_b, D_x Om_b, D_y Om_b at rows a, a+1; PEN: s/(1+s) at
// rows a-1 .. a+2, then dt sigma Uinf/(1+s) at the same rows.
template <int MODE>
__device__ __forceinline__ void roll_issue_aux(const Fields<float>& f0, const RollShape& rs, RollPos p, float* aux) {
    if (!RollArrays<MODE>::AUX || p.unit >= rs.nunits || p.s == 0) return;
    constexpr bool PEN = RollArrays<MODE>::PEN;
    const int m = p.unit / rs.upm, grp = p.unit % rs.upm;
    const size_t so = roll_off(f0, m).so;
    const int nx = f0.nx, ny = f0.ny, nq = nx >> 2;   // 16-byte chunks per row
    const int lognq = f0.logx - 2;
#pragma unroll 1
    for (int e = threadIdx.x; e < rs.G * nq; e += blockDim.x) {
        const int c = e & (nq - 1), g = e >> lognq;
        const int a = (grp * rs.G + g) * rs.R + 2 * (p.s - 1);
        float* dst = aux + (size_t)g * 8 * nx + 4 * c;
#pragma unroll
        for (int row = 0; row < 8; ++row) {
            const float* src;
            int r;
            if (PEN) {
                src = (row < 4 ? f0.cS : f0.cG) + so;
                r = (a - 1 + (row & 3) + ny) & (ny - 1);
            } else {
                const int arr = row >> 1;
                src = (arr == 0 ? f0.Ub : arr == 1 ? f0.Vb : arr == 2 ? f0.DxOb : f0.DyOb) + so;
                r = a + (row & 1);
            }
            cp_async16(dst + (size_t)row * nx, src + (size_t)r * nx + 4 * c);
        }
    }
}

// z = A + i B as a length-nx sequence from the packed half-spectra A, B
// (slot 0 holds X[0] in .x and X[nx/2] in .y)
__device__ __forceinline__ void roll_unpack(float2* z, int k, int nx, float2 A, float2 B) {
    if (k == 0) {
        z[0] = mk<float>(A.x, B.x);
        z[sw<float>(nx >> 1)] = mk<float>(A.y, B.y);
    } else {
        z[sw<float>(k)] = mk<float>(A.x - B.y, A.y + B.x);
        z[sw<float>(nx - k)] = mk<float>(A.x + B.y, B.x - A.y);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kRollThreads, 1) k_row_roll(Fields<float> f0, RollShape rs, bool sfd) {
    constexpr bool PEN = RollArrays<MODE>::PEN;
    constexpr bool AUX = RollArrays<MODE>::AUX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = f0.nx, nh = f0.nxh, ny = f0.ny, G = rs.G;
    const int nxp = padded_len(nx, 2);   // slots of one sequence (sw<float> pads)
    // [g][5][nxp]: ring slots 0..2, M0, M1
    float2* seqs = reinterpret_cast<float2*>(smem_raw);
    float4* stage = reinterpret_cast<float4*>(seqs + (size_t)G * 5 * nxp);   // [g][3][nx/2]
    float* aux = reinterpret_cast<float*>(stage + (size_t)G * 3 * nh);        // [g][8][nx]
    auto seq = [=](int g, int slot) { return seqs + ((size_t)g * 5 + slot) * nxp; };

    RollPos cur = roll_first(f0, rs);
    roll_issue_spectra<MODE>(f0, rs, cur, stage);
    cp_async_commit();
    roll_issue_aux<MODE>(f0, rs, cur, aux);
    cp_async_commit();
    while (cur.unit < rs.nunits) {
        const RollPos nxt = roll_next(f0, rs, cur);
        const int s = cur.s;
        cp_async_wait1();   // the spectra of this step
        __syncthreads();
        {
            const int ring_slot = (s + 1) % 3;
#pragma unroll 1
            for (int e = threadIdx.x; e < G * nh; e += blockDim.x) {
                const int k = e & (nh - 1), g = e >> (f0.logx - 1);
                const float4* st = stage + (size_t)g * 3 * nh + k;
                if (s == 0) {
                    for (int q = 0; q < 2; ++q) {
                        const float4 v = st[(size_t)q * nh];
                        roll_unpack(seq(g, q), k, nx, mk<float>(v.x, v.y), mk<float>(v.z, v.w));
                    }
                } else {
                    const float4 v0 = st[0], v1 = st[nh], v2 = st[2 * (size_t)nh];
                    roll_unpack(seq(g, ring_slot), k, nx, mk<float>(v0.x, v0.y), mk<float>(v0.z, v0.w));
                    if (PEN) {   // omega* and v* row pairs
                        roll_unpack(seq(g, 3), k, nx, mk<float>(v1.x, v1.y), mk<float>(v1.z, v1.w));
                        roll_unpack(seq(g, 4), k, nx, mk<float>(v2.x, v2.y), mk<float>(v2.z, v2.w));
                    } else {     // rows a and a+1 of (u', v)
                        roll_unpack(seq(g, 3), k, nx, mk<float>(v1.x, v1.y), mk<float>(v2.x, v2.y));
                        roll_unpack(seq(g, 4), k, nx, mk<float>(v1.z, v1.w), mk<float>(v2.z, v2.w));
                    }
                }
            }
        }
        __syncthreads();   // staging consumed: refill it with the next step's spectra
        roll_issue_spectra<MODE>(f0, rs, nxt, stage);
        cp_async_commit();
        {
            // s = 0: ring pairs -1 and 0 of every strip; s >= 1: ring pair s,
            // then the two sequences of row pair s - 1
            const int rs_slot = (s + 1) % 3, first = (s == 0);
            fft_smem_seqs<true, float, 3>(
                [=](int q) {
                    if (first) return seq(q >> 1, q & 1);
                    const int g = q / 3, w = q - 3 * g;
                    return seq(g, w == 0 ? rs_slot : 2 + w);
                },
                f0.logx, (first ? 2 : 3) * G, f0.twx[3]);
        }
        cp_async_wait1();   // the per-row operands of this step
        __syncthreads();
        if (s > 0) {
            const int t = s - 1;
            const int m = cur.unit / rs.upm, grp = cur.unit % rs.upm;
            const RollOff o = roll_off(f0, m);
            const float idx2 = f0.idx2, idy2 = f0.idy2, Uinf = f0.Uinf;
            const float cx = idx2 / (float)nx, cy = idy2 / (float)nx;   // 1/nx: exact
            const int sm = t % 3, s0 = (t + 1) % 3, sp = (t + 2) % 3;
#pragma unroll 1
            for (int e = threadIdx.x; e < G * nx; e += blockDim.x) {
                const int i = e & (nx - 1), g = e >> f0.logx;
                const int ip = (i + 1) & (nx - 1), im = (i - 1) & (nx - 1);
                const float2* Rm = seq(g, sm);   // pair t-1: rows a-2, a-1
                const float2* R0 = seq(g, s0);   // pair t:   rows a, a+1
                const float2* Rp = seq(g, sp);   // pair t+1: rows a+2, a+3
                float2* M0 = seq(g, 3);
                const float2* M1 = seq(g, 4);
                const float* ax = aux + (size_t)g * 8 * nx;
                const int a = (grp * G + g) * rs.R + 2 * t;
                float v0, v1;
                if (!PEN) {
                    // omega from the unnormalised inverse transform of its x-spectrum
                    const float2 rc = R0[sw<float>(i)], rpi = R0[sw<float>(ip)], rmi = R0[sw<float>(im)];
                    const float dxw0 = (rpi.x - rmi.x) * cx, dxw1 = (rpi.y - rmi.y) * cx;
                    const float dyw0 = (rc.y - Rm[sw<float>(i)].y) * cy;
                    const float dyw1 = (Rp[sw<float>(i)].x - rc.x) * cy;
                    const float2 uv0 = M0[sw<float>(i)], uv1 = M1[sw<float>(i)];
                    if (MODE == FWD_RHS_NL) {
                        v0 = -((Uinf + uv0.x) * dxw0 + uv0.y * dyw0);
                        v1 = -((Uinf + uv1.x) * dxw1 + uv1.y * dyw1);
                    } else {
                        v0 = -(ax[0 * nx + i] * dxw0 + ax[2 * nx + i] * dyw0 + uv0.x * ax[4 * nx + i] +
                               uv0.y * ax[6 * nx + i]);
                        v1 = -(ax[1 * nx + i] * dxw1 + ax[3 * nx + i] * dyw1 + uv1.x * ax[5 * nx + i] +
                               uv1.y * ax[7 * nx + i]);
                    }
                } else {
                    const float U = (MODE == FWD_PEN_NL) ? Uinf : 0.f;
                    const float* cS = ax;          // rows a-1 .. a+2
                    const float* cG = ax + 4 * nx;
                    const float2 um = Rm[sw<float>(i)], u0 = R0[sw<float>(i)], up = Rp[sw<float>(i)];
                    float dum1 = -cS[0 * nx + i] * (U + um.y);   // row a-1
                    float du0 = -cS[1 * nx + i] * (U + u0.x);    // row a
                    float du1 = -cS[2 * nx + i] * (U + u0.y);    // row a+1
                    float du2 = -cS[3 * nx + i] * (U + up.x);    // row a+2
                    if (MODE == FWD_PEN_NL) {
                        dum1 += cG[0 * nx + i];
                        du0 += cG[1 * nx + i];
                        du1 += cG[2 * nx + i];
                        du2 += cG[3 * nx + i];
                    }
                    const float2 vp = M1[sw<float>(ip)], vm = M1[sw<float>(im)];
                    const float dvp0 = -cS[1 * nx + ip] * vp.x, dvm0 = -cS[1 * nx + im] * vm.x;
                    const float dvp1 = -cS[2 * nx + ip] * vp.y, dvm1 = -cS[2 * nx + im] * vm.y;
                    const float2 ws = M0[sw<float>(i)];
                    v0 = ws.x + (dvp0 - dvm0) * idx2 - (du1 - dum1) * idy2;
                    v1 = ws.y + (dvp1 - dvm1) * idx2 - (du2 - du0) * idy2;
                    const size_t c0 = (size_t)a * nx + i, c1 = c0 + nx;
                    if (sfd) {
                        float* Y = f0.Y + o.fo;
                        const float y0 = Y[c0], y1 = Y[c1];
                        const float d0 = v0 - y0, d1 = v1 - y1;
                        Y[c0] = y0 + f0.sfd_k2 * d0;
                        Y[c1] = y1 + f0.sfd_k2 * d1;
                        v0 = v0 - f0.sfd_k1 * d0;
                        v1 = v1 - f0.sfd_k1 * d1;
                    }
                    if (rs.write_w) {
                        f0.W[o.fo + c0] = v0;
                        f0.W[o.fo + c1] = v1;
                    }
                }
                M0[sw<float>(i)] = mk<float>(v0, v1);
            }
            const bool fwd = !PEN || rs.do_fft;
            if (fwd) {
                __syncthreads();
                fft_smem_seqs<false, float, 3>([=](int g) { return seq(g, 3); }, f0.logx, G, f0.twx[3]);
                float2* dst = (PEN ? f0.X1 : f0.X4) + o.co;
    #pragma unroll 1
                for (int e = threadIdx.x; e < G * nh; e += blockDim.x) {
                    const int k = e & (nh - 1), g = e >> (f0.logx - 1);
                    const int a = (grp * G + g) * rs.R + 2 * t;
                    const float2* z = seq(g, 3);
                    float2 A, B;
                    if (k == 0) {
                        const float2 z0 = z[0], zn = z[sw<float>(nh)];
                        A = mk<float>(z0.x, zn.x);
                        B = mk<float>(z0.y, zn.y);
                    } else {
                        const float2 zk = z[sw<float>(k)];
                        const float2 zm = cconj(z[sw<float>(nx - k)]);
                        A = cscale(cadd(zk, zm), 0.5f);
                        B = cscale(cmul_mi(csub(zk, zm)), 0.5f);
                    }
                    PairIO<float>::store(dst + (size_t)k * ny + a, A, B);
                }
            }
        }
        __syncthreads();   // per-row operands and sequences consumed
        roll_issue_aux<MODE>(f0, rs, nxt, aux);
        cp_async_commit();
        cur = nxt;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

}  // namespace nsstab
