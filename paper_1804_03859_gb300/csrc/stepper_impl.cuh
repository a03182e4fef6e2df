// The vorticity-streamfunction time-stepper: kernels and host driver.
//
// One time step (nonlinear or linearised, Sec. 3, Eqs. 28-30) is six
// kernels, alternating row passes (x-direction FFT of two real rows packed
// into one complex transform, with the finite-difference stencil fused into
// the forward pass) and column passes (y-direction FFT with the spectral
// diagonal operators fused between the forward and inverse transforms):
//
//   col_poisson   X1 (x-spectrum of omega)  -> Wh = FFT2(omega), X2 = x-spectrum of psi
//   row_inverse   X2                        -> P = psi
//   row_forward   RHS: W, P (+ base)        -> X1 = x-spectrum of N
//   col_update    X1, Wh, Nh                -> Nh = FFT2(N), X1/X2 = x-spectra of omega*, psi*
//   row_inverse   X1, X2                    -> W = omega*, P = psi*
//   row_forward   PEN: W, P (+ SFD state Y) -> W = omega^{n+1}, X1 = its x-spectrum
//
// FP32 steppers take three measures against error that a time-stepper
// would otherwise accumulate over hundreds of steps:
//  * they carry the velocity instead of the streamfunction: the column
//    passes form the x-spectra of u' = D_y psi and v = -D_x psi by
//    multiplying psi^ with the centred-difference symbols i sin(k h)/h (the
//    same discrete operator as the stencil on psi), and the inverse row
//    passes produce U, V (and W).  The stencil on a rounded psi loses about
//    log2(|psi| / (h |D psi|)) bits to cancellation (a per-step error near
//    7e-6 at 512x256); the spectral form keeps the velocity error at the
//    rounding of the velocity itself;
//  * the Crank-Nicolson factor A = (1 + nu dt lam/2)/(1 - nu dt lam/2),
//    within 1e-3 of 1 for the modes that carry the flow, is stored as
//    A - 1: an FP32 A is a fixed relative error of up to 3e-8 applied at
//    every step, which grows linearly over a run;
//  * their transforms split each twiddle into hi + lo (fft.cuh), for the
//    same reason.
// Together these take the FP32 propagator of 200 steps from about 1e-5 to
// about 1e-6 relative to FP64.  The FP64 and double-float steppers keep psi,
// the stencil and plain tables (their rounding is far below the parity bar),
// with 1.5x fewer row transforms.
//
// Layouts: physical fields [ny][nx] (x fastest); every spectral array is
// stored column-major [kx][ky] over the nx/2 packed x-wavenumbers, so the
// column passes read and write contiguous columns.  The x-transform of a
// real row is packed into nx/2 complex slots: slot 0 holds X[0] (real) in
// .x and X[nx/2] (real) in .y.  In the column passes the packed kx = 0
// column is the y-transform of (X0 + i XN); the spectral operators act on it
// through its Hermitian halves (see apply_packed0).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include "fft.cuh"
#include "stepper.cuh"

namespace nsstab {

enum RowMode { FWD_PLAIN = 0, FWD_RHS_NL = 1, FWD_RHS_LIN = 2, FWD_PEN_NL = 3, FWD_PEN_LIN = 4 };

// The FP32 stepper's accuracy measures (see the file comment): velocities
// in place of psi, and the Crank-Nicolson factor stored as A - 1.  (Its
// transforms also split twiddles into hi + lo; see fft.cuh.)
template <class T> constexpr bool kF32 = std::is_same<T, float>::value;

template <class T> struct Fields {
    int nx, ny, nxh, logx, logy;
    int bper;              // members per parameter set (member m uses set m / bper)
    size_t fs, cs, ts;     // member strides: physical field, spectrum, operator table
    const unsigned char* active;   // per-member flag: inactive members skip every kernel
    T idx2, idy2;          // 1/(2 dx), 1/(2 dy)
    T Uinf;
    T scale;               // 1/(nx ny), the normalisation of the inverse transform
    T sfd_k1, sfd_k2;      // dt*chi_sfd, dt/Delta
    T* W;                  // omega (physical)
    T* P;                  // psi (physical)
    T* U; T* V;            // u' = D_y psi, v = -D_x psi (physical; kVel steppers)
    T* Y;                  // SFD filtered state
    const T* cS;           // s/(1+s), s = dt (chi/eta + sigma)
    const T* cG;           // dt sigma Uinf / (1+s)
    const T* Ub; const T* Vb; const T* DxOb; const T* DyOb;   // base-derived fields
    Cx<T>* X1; Cx<T>* X2;  // x-spectral, y-physical [kx][y]
    Cx<T>* X3;             // x-spectrum of v (kVel steppers)
    Cx<T>* X4;             // x-spectrum of N written by the fused row pass (FP32)
    const Cx<T>* XN;       // x-spectrum of N read by k_col_update (X1, or X4)
    Cx<T>* Wh; Cx<T>* Nh;  // full spectra [kx][ky]
    const T* tA; const T* tB; const T* tP;   // spectral operator tables [nxh+1][ny]
    const T* tDx; const T* tDy;              // sin(2 pi kx/nx)/dx [nxh+1], sin(2 pi ky/ny)/dy [ny]
    const Cx<T>* twx[4]; const Cx<T>* twy[4];   // per-pass twiddle tables for LE = 1, 2, 3
};

// Offset the member-dependent pointers to member m (and its parameter
// set).  Returns false for an inactive member: its blocks return
// at once, so independent solves of a batch can drop out or idle.
template <class T> __device__ __forceinline__ bool member_view_at(Fields<T>& f, int m) {
    if (f.active && !f.active[m]) return false;
    const int set = m / f.bper;
    const size_t fo = (size_t)m * f.fs, co = (size_t)m * f.cs, so = (size_t)set * f.fs, to = (size_t)set * f.ts;
    f.W += fo;
    f.P += fo;
    if (f.Y) f.Y += fo;
    f.X1 += co;
    f.X2 += co;
    f.XN += co;
    if (kF32<T>) {
        f.U += fo;
        f.V += fo;
        f.X3 += co;
        f.X4 += co;
    }
    f.Wh += co;
    f.Nh += co;
    f.cS += so;
    f.cG += so;
    if (f.Ub) {
        f.Ub += so;
        f.Vb += so;
        f.DxOb += so;
        f.DyOb += so;
    }
    f.tA += to;
    f.tB += to;
    return true;
}

template <class T> __device__ __forceinline__ bool member_view(Fields<T>& f) { return member_view_at(f, blockIdx.y); }

// Diagonal operators at (kx, ky), kx in [0, nx/2]: Crank-Nicolson A = a/b
// (FP32 steppers: A - 1), B = dt/b (both times the 1/(nx ny) of the inverse
// transform) and the
// inverse Laplacian P = -1/lam (zero for the mean mode), read from tables
// computed on the host in FP64 and rounded once to the stepper's precision
// (a division costs ~10 FP64 instructions on GB300, and evaluating them in
// FP32 on the device adds several roundings that show in the FP32
// eigenvalues).
template <class T> struct SpecOp {
    __device__ static __forceinline__ void ab(const Fields<T>& f, int kx, int ky, T& A, T& B) {
        const size_t g = (size_t)kx * f.ny + ky;
        A = f.tA[g];
        B = f.tB[g];
    }
    __device__ static __forceinline__ T p(const Fields<T>& f, int kx, int ky) { return f.tP[(size_t)kx * f.ny + ky]; }
};

// ------------------------------------------------------------ point values

// Value of row j at column i for the forward row pass.  PEN modes return the
// new vorticity (and the new SFD filter value in *y_new) without storing
// them, so that a thread can issue all of its loads before its first store.
template <class T, int MODE>
__device__ __forceinline__ T row_value(const Fields<T>& f, int i, int j, bool sfd, T* y_new) {
    const int nx = f.nx, ny = f.ny;
    const int ip = (i + 1) & (nx - 1), im = (i - 1) & (nx - 1);
    const int jp = (j + 1) & (ny - 1), jm = (j - 1) & (ny - 1);
    const size_t c = (size_t)j * nx + i;
    if (MODE == FWD_PLAIN) {
        return f.W[c];
    } else if (MODE == FWD_RHS_NL || MODE == FWD_RHS_LIN) {
        const T* W = f.W;
        const T dxw = (W[(size_t)j * nx + ip] - W[(size_t)j * nx + im]) * f.idx2;
        const T dyw = (W[(size_t)jp * nx + i] - W[(size_t)jm * nx + i]) * f.idy2;
        T up, vp;   // u' = D_y psi, v = -D_x psi at (i, j)
        if (kF32<T>) {
            up = f.U[c];
            vp = f.V[c];
        } else {
            const T* P = f.P;
            up = (P[(size_t)jp * nx + i] - P[(size_t)jm * nx + i]) * f.idy2;
            vp = -((P[(size_t)j * nx + ip] - P[(size_t)j * nx + im]) * f.idx2);
        }
        if (MODE == FWD_RHS_NL) {
            const T u = f.Uinf + up;
            return -(u * dxw + vp * dyw);
        } else {
            // N' = -(U_b D_x w + V_b D_y w + u' D_x Om_b + v' D_y Om_b)
            return -(f.Ub[c] * dxw + f.Vb[c] * dyw + up * f.DxOb[c] + vp * f.DyOb[c]);
        }
    } else {
        // omega^{n+1} = omega* + D_x dv - D_y du with the implicit Brinkman +
        // fringe velocity correction du = cG - cS u*, dv = -cS v*.
        const T U = (MODE == FWD_PEN_NL) ? f.Uinf : T(0);
        const size_t rj = (size_t)j * nx;
        const size_t cp = (size_t)jp * nx + i, cm = (size_t)jm * nx + i;
        // v* at (i+1, j) and (i-1, j), u* at (i, j+1) and (i, j-1)
        const T* P = f.P;
        T vp, vm, up, um;
        if (kF32<T>) {
            vp = f.V[rj + ip];
            vm = f.V[rj + im];
        } else {
            const int ipp = (i + 2) & (nx - 1), imm = (i - 2) & (nx - 1);
            vp = -((P[rj + ipp] - P[rj + i]) * f.idx2);
            vm = -((P[rj + i] - P[rj + imm]) * f.idx2);
        }
        const T dvp = -f.cS[rj + ip] * vp;
        const T dvm = -f.cS[rj + im] * vm;
        if (kF32<T>) {
            up = U + f.U[cp];
            um = U + f.U[cm];
        } else {
            const int jpp = (j + 2) & (ny - 1), jmm = (j - 2) & (ny - 1);
            up = U + (P[(size_t)jpp * nx + i] - P[c]) * f.idy2;
            um = U + (P[c] - P[(size_t)jmm * nx + i]) * f.idy2;
        }
        T dup = -f.cS[cp] * up;
        T dum = -f.cS[cm] * um;
        if (MODE == FWD_PEN_NL) {
            dup += f.cG[cp];
            dum += f.cG[cm];
        }
        T w = f.W[c] + (dvp - dvm) * f.idx2 - (dup - dum) * f.idy2;
        if (sfd) {
            const T y = f.Y[c];
            const T d = w - y;
            *y_new = y + f.sfd_k2 * d;
            w = w - f.sfd_k1 * d;
        }
        return w;
    }
}

// -------------------------------------------------------------- row kernels

// Forward x-transform of RP row pairs per block, with the row values made by
// MODE.  Writes the packed half-spectra to X1 ([kx][y]) when do_fft.
// Register budget: blocks of up to 512 threads at 8 elements per thread (the
// largest rows, nx = 4096, need 512), up to 1024 otherwise.
#define NS_FFT_BOUNDS __launch_bounds__(LE == 3 ? 512 : 1024)

template <class T, int MODE, int LE>
__device__ __forceinline__ void row_forward_body(const Fields<T>& f, int bx, int RP, int logRP, bool sfd,
                                                 bool do_fft) {
    using C = Cx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int nx = f.nx, S = seq_stride(nx, RP, (int)sizeof(C) / 4);
    const int pair0 = bx * RP;
    constexpr int E = 1 << LE;   // RP*nx values over RP*nx/E threads: exactly E each
    constexpr bool PEN = (MODE == FWD_PEN_NL || MODE == FWD_PEN_LIN);
    T va[E], vb[E], ya[PEN ? E : 1], yb[PEN ? E : 1];
#pragma unroll
    for (int it = 0; it < E; ++it) {
        const int e = threadIdx.x + it * blockDim.x;
        const int p = e >> f.logx, i = e & (nx - 1);
        const int j0 = 2 * (pair0 + p);
        va[it] = row_value<T, MODE>(f, i, j0, sfd, &ya[PEN ? it : 0]);
        vb[it] = row_value<T, MODE>(f, i, j0 + 1, sfd, &yb[PEN ? it : 0]);
    }
#pragma unroll
    for (int it = 0; it < E; ++it) {
        const int e = threadIdx.x + it * blockDim.x;
        const int p = e >> f.logx, i = e & (nx - 1);
        const int j0 = 2 * (pair0 + p);
        if (PEN) {
            const size_t c = (size_t)j0 * nx + i;
            f.W[c] = va[it];
            f.W[c + nx] = vb[it];
            if (sfd) {
                f.Y[c] = ya[PEN ? it : 0];
                f.Y[c + nx] = yb[PEN ? it : 0];
            }
        }
        s[p * S + sw<T>(i)] = mk<T>(va[it], vb[it]);
    }
    if (!do_fft) return;
    __syncthreads();
    fft_smem<false, T, LE>(s, f.logx, S, RP, f.twx[LE]);
    // split Z = FFT(a + i b) into the half-spectra of a and b
    const int nh = nx >> 1;
#pragma unroll
    for (int it = 0; it < E / 2; ++it) {
        const int e = threadIdx.x + it * blockDim.x;
        const int p = e & (RP - 1), k = e >> logRP;
        const int j0 = 2 * (pair0 + p);
        const C* z = s + p * S;
        C A, B;
        if (k == 0) {
            const C z0 = z[0], zn = z[sw<T>(nh)];
            A = mk<T>(z0.x, zn.x);
            B = mk<T>(z0.y, zn.y);
        } else {
            const C zk = z[sw<T>(k)];
            const C zm = cconj(z[sw<T>(nx - k)]);
            A = cscale(cadd(zk, zm), T(0.5));
            B = cscale(cmul_mi(csub(zk, zm)), T(0.5));
        }
        PairIO<T>::store(f.X1 + (size_t)k * f.ny + j0, A, B);   // rows j0, j0+1 are adjacent
    }
}

template <class T, int MODE, int LE>
__global__ void NS_FFT_BOUNDS k_row_forward(Fields<T> f, int RP, int logRP, bool sfd, bool do_fft) {
    if (!member_view(f)) return;
    row_forward_body<T, MODE, LE>(f, blockIdx.x, RP, logRP, sfd, do_fft);
}

// What an inverse row pass transforms.  Each complex transform carries two
// real rows: either rows (2p, 2p+1) of one array (a "same" pass) or row p of
// two arrays.
enum InvIO {
    INV_PSI = 0,   // X2 row pairs -> P
    INV_WP = 1,    // X1 -> W, X2 -> P, row by row
    INV_UV = 2,    // X2 -> U, X3 -> V, row by row
    INV_WUV = 3,   // blocks over rows [0, ny): X1 -> W, X2 -> U; then X3 row pairs -> V
};

// Inverse x-transform of RP sequences per block, as selected by IO.
template <class T, int LE, int IO>
__device__ __forceinline__ void row_inverse_body(const Fields<T>& f, int bx, int RP, int logRP) {
    using C = Cx<T>;
    int pair0 = bx * RP;
    bool same = (IO == INV_PSI);
    const C* XA = (IO == INV_PSI || IO == INV_UV) ? f.X2 : f.X1;
    const C* XB = (IO == INV_UV) ? f.X3 : f.X2;
    T* dA = (IO == INV_PSI) ? f.P : (IO == INV_UV) ? f.U : f.W;
    T* dB = (IO == INV_UV) ? f.V : (IO == INV_WUV) ? f.U : f.P;
    if (IO == INV_WUV && pair0 >= f.ny) {   // RP divides ny/2: a block lies wholly in one part
        same = true;
        pair0 -= f.ny;
        XA = XB = f.X3;
        dA = dB = f.V;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int nx = f.nx, ny = f.ny, nh = nx >> 1, S = seq_stride(nx, RP, (int)sizeof(C) / 4);
    constexpr int E = 1 << LE;   // RP*nh spectra over RP*nx/E threads: E/2 each
    C Av[E / 2], Bv[E / 2];
#pragma unroll
    for (int it = 0; it < E / 2; ++it) {
        const int e = threadIdx.x + it * blockDim.x;
        const int p = e & (RP - 1), k = e >> logRP;
        const int ra = same ? 2 * (pair0 + p) : pair0 + p;
        if (same) {
            PairIO<T>::load(XA + (size_t)k * ny + ra, Av[it], Bv[it]);   // rows 2pr, 2pr+1 are adjacent
        } else {
            Av[it] = XA[(size_t)k * ny + ra];
            Bv[it] = XB[(size_t)k * ny + ra];
        }
    }
#pragma unroll
    for (int it = 0; it < E / 2; ++it) {
        const int e = threadIdx.x + it * blockDim.x;
        const int p = e & (RP - 1), k = e >> logRP;
        const C A = Av[it], B = Bv[it];
        C* z = s + p * S;
        if (k == 0) {
            z[0] = mk<T>(A.x, B.x);
            z[sw<T>(nh)] = mk<T>(A.y, B.y);
        } else {
            z[sw<T>(k)] = mk<T>(A.x - B.y, A.y + B.x);        // A + i B
            z[sw<T>(nx - k)] = mk<T>(A.x + B.y, B.x - A.y);   // conj(A) + i conj(B)
        }
    }
    __syncthreads();
    fft_smem<true, T, LE>(s, f.logx, S, RP, f.twx[LE]);
#pragma unroll
    for (int it = 0; it < E; ++it) {
        const int e = threadIdx.x + it * blockDim.x;
        const int p = e >> f.logx, i = e & (nx - 1);
        const int pr = pair0 + p;
        const int ra = same ? 2 * pr : pr;
        const int rb = same ? 2 * pr + 1 : pr;
        const C z = s[p * S + sw<T>(i)];
        dA[(size_t)ra * nx + i] = z.x;
        (same ? dA : dB)[(size_t)rb * nx + i] = z.y;
    }
}

template <class T, int LE, int IO>
__global__ void NS_FFT_BOUNDS k_row_inverse(Fields<T> f, int RP, int logRP) {
    if (!member_view(f)) return;
    row_inverse_body<T, LE, IO>(f, blockIdx.x, RP, logRP);
}

// ----------------------------------------------------------- column kernels

// Packed kx = 0 column: Z = FFT_y(X0 + i XN).  Applying real operators f0 to
// the kx = 0 part and fN to the kx = nx/2 part gives
//   Z'(ky) = (f0 + fN)/2 Z(ky) + (f0 - fN)/2 conj(Z(-ky)).
template <class C, class T>
__device__ __forceinline__ C apply_packed0(C z, C zm_conj, T f0, T fN) {
    return cadd(cscale(z, T(0.5) * (f0 + fN)), cscale(zm_conj, T(0.5) * (f0 - fN)));
}

// Forward y-transform of CP columns of X1, store Wh, psi^ = scale * tP * omega^,
// inverse y-transform into X2.  VEL: inverse y-transforms of
// u'^ = i sy psi^ into X2 and v^ = -i sx psi^ into X3 instead, with
// sy = sin(2 pi ky/ny)/dy, sx = sin(2 pi kx/nx)/dx, the symbols of the
// centred differences (zero at kx = 0 and kx = nx/2, so the packed column of
// v is zero; sy is odd in ky and acts alike on both halves of the packed
// column).
template <class T, int LE, bool VEL>
__device__ __forceinline__ void col_poisson_body(const Fields<T>& f, int bx, int CP, T scale) {
    using C = Cx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int ny = f.ny, logy = f.logy;
    const int S = seq_stride(ny, (ny >> LE) < 32 ? 32 / (ny >> LE) : 1, (int)sizeof(C) / 4);
    C* s2 = s + (size_t)CP * S;   // VEL: v^
    const int c0 = bx * CP;
    constexpr int E = 1 << LE;   // E elements per thread in each FFT pass
    // CP*ny values over blockDim threads: E each, or E/2 when the block has
    // twice the threads of one transform round (both inverse columns at once)
    const int EL = (CP << logy) / blockDim.x;
    {
        C v[E];
#pragma unroll
        for (int it = 0; it < E; ++it)
            if (it < EL) v[it] = f.X1[(size_t)c0 * ny + threadIdx.x + it * blockDim.x];
#pragma unroll
        for (int it = 0; it < E; ++it) {
            const int e = threadIdx.x + it * blockDim.x;
            if (it < EL) s[(e >> logy) * S + sw<T>(e & (ny - 1))] = v[it];
        }
    }
    __syncthreads();
    fft_smem<false, T, LE>(s, logy, S, CP, f.twy[LE]);
    for (int e = threadIdx.x; e < (CP << logy); e += blockDim.x) {
        const int c = e >> logy, k = e & (ny - 1);
        f.Wh[(size_t)(c0 + c) * ny + k] = s[c * S + sw<T>(k)];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (CP << logy); e += blockDim.x) {
        const int c = e >> logy, k = e & (ny - 1);
        const int kx = c0 + c;
        C* z = s + c * S;
        if (kx != 0) {
            const C ps = cscale(z[sw<T>(k)], scale * SpecOp<T>::p(f, kx, k));
            if (VEL) {
                z[sw<T>(k)] = cscale(cmul_pi(ps), f.tDy[k]);
                s2[c * S + sw<T>(k)] = cscale(cmul_mi(ps), f.tDx[kx]);
            } else {
                z[sw<T>(k)] = ps;
            }
        } else if (k <= (ny >> 1)) {
            const int km = (ny - k) & (ny - 1);
            const T f0 = scale * SpecOp<T>::p(f, 0, k), fN = scale * SpecOp<T>::p(f, f.nxh, k);
            const C zk = z[sw<T>(k)], zm = z[sw<T>(km)];
            C pk = apply_packed0(zk, cconj(zm), f0, fN);
            C pm = apply_packed0(zm, cconj(zk), f0, fN);
            if (VEL) {
                pk = cscale(cmul_pi(pk), f.tDy[k]);
                pm = cscale(cmul_pi(pm), f.tDy[km]);
                s2[sw<T>(k)] = mk<T>(T(0), T(0));
                s2[sw<T>(km)] = mk<T>(T(0), T(0));
            }
            z[sw<T>(k)] = pk;
            if (km != k) z[sw<T>(km)] = pm;
        }
    }
    __syncthreads();
    fft_smem<true, T, LE>(s, logy, S, VEL ? 2 * CP : CP, f.twy[LE]);
    for (int e = threadIdx.x; e < (CP << logy); e += blockDim.x) {
        const int c = e >> logy, j = e & (ny - 1);
        const size_t g = (size_t)(c0 + c) * ny + j;
        f.X2[g] = s[c * S + sw<T>(j)];
        if (VEL) f.X3[g] = s2[c * S + sw<T>(j)];
    }
}

template <class T, int LE, bool VEL>
__global__ void NS_FFT_BOUNDS k_col_poisson(Fields<T> f, int CP, T scale) {
    if (!member_view(f)) return;
    col_poisson_body<T, LE, VEL>(f, blockIdx.x, CP, scale);
}

// Forward y-transform of N (x-spectra in XN: X1, or X4 after the fused FP32
// row pass); AB2/AB1 + Crank-Nicolson update
//   omega*^ = tA omega^ + tB (c1 N^n + c0 N^{n-1}),  psi*^ = tP omega*^
// (tA, tB carry the 1/(nx ny) of the inverse transform); Nh <- N^n; inverse
// y-transforms of omega*^ -> X1 and psi*^ -> X2 (kVel: u*'^ -> X2 and
// v*^ -> X3, as in k_col_poisson).
template <class T, int LE>
__device__ __forceinline__ void col_update_body(const Fields<T>& f, int bx, int CP, T c1, T c0, bool first) {
    using C = Cx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s1 = reinterpret_cast<C*>(smem_raw);
    const int ny = f.ny, logy = f.logy;
    const int S = seq_stride(ny, (ny >> LE) < 32 ? 32 / (ny >> LE) : 1, (int)sizeof(C) / 4);
    C* s2 = s1 + (size_t)CP * S;   // omega^ in, psi*^ out
    C* s3 = s2 + (size_t)CP * S;   // N^{n-1} in
    const int c0i = bx * CP;
    constexpr int E = 1 << LE;   // E elements per thread in each FFT pass
    // CP*ny values over blockDim threads: E each, or E/2 when the block has
    // twice the threads of one transform round (the inverse transforms of
    // omega*, psi* (and v*) then run side by side)
    const int EL = (CP << logy) / blockDim.x;
    // all three input columns are read at once (one wait for the whole block)
    {
        C a[E], b[E], c3[E];
#pragma unroll
        for (int it = 0; it < E; ++it) {
            if (it >= EL) continue;
            const size_t g = (size_t)c0i * ny + threadIdx.x + it * blockDim.x;
            a[it] = f.XN[g];
            b[it] = f.Wh[g];
            if (!first) c3[it] = f.Nh[g];
        }
#pragma unroll
        for (int it = 0; it < E; ++it) {
            if (it >= EL) continue;
            const int e = threadIdx.x + it * blockDim.x;
            const int o = (e >> logy) * S + sw<T>(e & (ny - 1));
            s1[o] = a[it];
            s2[o] = b[it];
            if (!first) s3[o] = c3[it];
        }
    }
    __syncthreads();
    fft_smem<false, T, LE>(s1, logy, S, CP, f.twy[LE]);
    for (int e = threadIdx.x; e < (CP << logy); e += blockDim.x) {
        const int c = e >> logy, k = e & (ny - 1);
        const int kx = c0i + c;
        const size_t g = (size_t)kx * ny + k;
        C* z1 = s1 + c * S;
        C* z2 = s2 + c * S;
        C* z3 = s3 + c * S;
        if (kx != 0) {
            const C nn = z1[sw<T>(k)];
            const C r = first ? cscale(nn, c1) : cadd(cscale(nn, c1), cscale(z3[sw<T>(k)], c0));
            f.Nh[g] = nn;
            T A, B;
            SpecOp<T>::ab(f, kx, k, A, B);
            C ws;
            if constexpr (kF32<T>) {   // tA = scale (A - 1): the small terms first, one rounding at the end
                const C wv = z2[sw<T>(k)];
                const C t = cadd(cscale(wv, A), cscale(r, B));
                ws = mk<T>(__fmaf_rn(wv.x, f.scale, t.x), __fmaf_rn(wv.y, f.scale, t.y));
            } else {
                ws = cadd(cscale(z2[sw<T>(k)], A), cscale(r, B));
            }
            z1[sw<T>(k)] = ws;
            const C ps = cscale(ws, SpecOp<T>::p(f, kx, k));
            if (kF32<T>) {
                z2[sw<T>(k)] = cscale(cmul_pi(ps), f.tDy[k]);
                z3[sw<T>(k)] = cscale(cmul_mi(ps), f.tDx[kx]);
            } else {
                z2[sw<T>(k)] = ps;
            }
        } else if (k <= (ny >> 1)) {
            const int km = (ny - k) & (ny - 1);
            const C nk = z1[sw<T>(k)], nm = z1[sw<T>(km)];
            C rk = cscale(nk, c1), rm = cscale(nm, c1);
            if (!first) {
                rk = cadd(rk, cscale(z3[sw<T>(k)], c0));
                rm = cadd(rm, cscale(z3[sw<T>(km)], c0));
            }
            f.Nh[k] = nk;
            f.Nh[km] = nm;
            T A0k, B0k, ANk, BNk, A0m, B0m, ANm, BNm;
            SpecOp<T>::ab(f, 0, k, A0k, B0k);
            SpecOp<T>::ab(f, f.nxh, k, ANk, BNk);
            SpecOp<T>::ab(f, 0, km, A0m, B0m);
            SpecOp<T>::ab(f, f.nxh, km, ANm, BNm);
            const C wk = z2[sw<T>(k)], wm = z2[sw<T>(km)];
            C wsk = cadd(apply_packed0(wk, cconj(wm), A0k, ANk), apply_packed0(rk, cconj(rm), B0k, BNk));
            C wsm = cadd(apply_packed0(wm, cconj(wk), A0m, ANm), apply_packed0(rm, cconj(rk), B0m, BNm));
            if constexpr (kF32<T>) {   // plus scale * omega^ (tA holds scale (A - 1))
                wsk = mk<T>(__fmaf_rn(wk.x, f.scale, wsk.x), __fmaf_rn(wk.y, f.scale, wsk.y));
                wsm = mk<T>(__fmaf_rn(wm.x, f.scale, wsm.x), __fmaf_rn(wm.y, f.scale, wsm.y));
            }
            z1[sw<T>(k)] = wsk;
            z1[sw<T>(km)] = wsm;
            C pk = apply_packed0(wsk, cconj(wsm), SpecOp<T>::p(f, 0, k), SpecOp<T>::p(f, f.nxh, k));
            C pm = apply_packed0(wsm, cconj(wsk), SpecOp<T>::p(f, 0, km), SpecOp<T>::p(f, f.nxh, km));
            if (kF32<T>) {
                pk = cscale(cmul_pi(pk), f.tDy[k]);
                pm = cscale(cmul_pi(pm), f.tDy[km]);
                z3[sw<T>(k)] = mk<T>(T(0), T(0));
                z3[sw<T>(km)] = mk<T>(T(0), T(0));
            }
            z2[sw<T>(k)] = pk;
            z2[sw<T>(km)] = pm;
        }
    }
    __syncthreads();
    fft_smem<true, T, LE>(s1, logy, S, (kF32<T> ? 3 : 2) * CP, f.twy[LE]);
    for (int e = threadIdx.x; e < (CP << logy); e += blockDim.x) {
        const int c = e >> logy, j = e & (ny - 1);
        const size_t g = (size_t)(c0i + c) * ny + j;
        f.X1[g] = s1[c * S + sw<T>(j)];
        f.X2[g] = s2[c * S + sw<T>(j)];
        if (kF32<T>) f.X3[g] = s3[c * S + sw<T>(j)];
    }
}

template <class T, int LE>
__global__ void NS_FFT_BOUNDS k_col_update(Fields<T> f, int CP, T c1, T c0, bool first) {
    if (!member_view(f)) return;
    col_update_body<T, LE>(f, blockIdx.x, CP, c1, c0, first);
}

// ------------------------------------------------------- pointwise kernels

// Base-derived fields of parameter set blockIdx.y, from Omega_b and Psi_b
// (kVel: the base velocity) held in member slot blockIdx.y of W and P (U, V).
template <class T>
__global__ void k_base_fields(Fields<T> f, T* Ub, T* Vb, T* DxOb, T* DyOb) {
    const size_t n = (size_t)f.nx * f.ny;
    const size_t off = (size_t)blockIdx.y * f.fs;
    const T* P = f.P + off;   // Psi_b
    const T* W = f.W + off;   // Omega_b
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(c & (f.nx - 1));
        const int j = (int)(c >> f.logx);
        const int ip = (i + 1) & (f.nx - 1), im = (i - 1) & (f.nx - 1);
        const int jp = (j + 1) & (f.ny - 1), jm = (j - 1) & (f.ny - 1);
        if (kF32<T>) {   // u', v of the base in U, V
            Ub[off + c] = f.Uinf + f.U[off + c];
            Vb[off + c] = f.V[off + c];
        } else {
            Ub[off + c] = f.Uinf + (P[(size_t)jp * f.nx + i] - P[(size_t)jm * f.nx + i]) * f.idy2;
            Vb[off + c] = -((P[(size_t)j * f.nx + ip] - P[(size_t)j * f.nx + im]) * f.idx2);
        }
        DxOb[off + c] = (W[(size_t)j * f.nx + ip] - W[(size_t)j * f.nx + im]) * f.idx2;
        DyOb[off + c] = (W[(size_t)jp * f.nx + i] - W[(size_t)jm * f.nx + i]) * f.idy2;
    }
}

// dst[m] <- src[m] (FP64 -> T) for the members with a non-null source
template <class T>
__global__ void k_gather(const double* const* __restrict__ src, T* __restrict__ dst, size_t n, size_t fs) {
    const double* s = src[blockIdx.y];
    if (!s) return;
    T* d = dst + (size_t)blockIdx.y * fs;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
        d[c] = (T)s[c];
}

// dst[m] <- src[m] (T -> FP64) for the members with a non-null destination
template <class T>
__global__ void k_scatter(const T* __restrict__ src, double* const* __restrict__ dst, size_t n, size_t fs) {
    double* d = dst[blockIdx.y];
    if (!d) return;
    const T* s = src + (size_t)blockIdx.y * fs;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
        d[c] = (double)s[c];
}

// partial[m][b] = sum over block b's share of (a - b)^2 of member m, in FP64
template <class T>
__global__ void k_diff_sumsq(const T* __restrict__ a, const T* __restrict__ b, size_t n, size_t fs, double* partial) {
    a += (size_t)blockIdx.y * fs;
    b += (size_t)blockIdx.y * fs;
    partial += (size_t)blockIdx.y * gridDim.x;
    double acc = 0.0;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const double d = (double)a[c] - (double)b[c];
        acc += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = acc;
    }
}

}  // namespace nsstab

#include "rowroll.cuh"   // fused FP32 row passes (uses Fields, row modes and the FFT above)

namespace nsstab {

// ------------------------------------------------------------- host side

// One launch configuration: `per` sequences (row pairs or columns) per
// block, 2^le elements per thread in the FFT passes; grid.y = members.
struct Launch {
    int blocks = 0, threads = 0, per = 0, logper = 0, le = 3;
    int tm = 1;            // column passes: threads per block = tm x one transform round
    size_t smem = 0;
    bool ok = false;
};

// the six kernels of a step, in order
enum KernelId { KCOLP = 0, KINVP = 1, KFWDR = 2, KCOLU = 3, KINVR = 4, KFWDP = 5 };
template <class T> int max_threads_for(int kid, int le);

static const int kRedBlocks = 64;           // partial sums per member
static const int kPtBlocks = 152;           // grid.x of the pointwise kernels
static const double kPi = 3.14159265358979323846;
static const int kGraphChunk = 256;         // time steps per captured graph
static const size_t kMaxSmem = 200 * 1024;

#define K_FWD_PLAIN(le) k_row_forward<T, FWD_PLAIN, le>
#define K_FWD_RNL(le) k_row_forward<T, FWD_RHS_NL, le>
#define K_FWD_RLIN(le) k_row_forward<T, FWD_RHS_LIN, le>
#define K_FWD_PNL(le) k_row_forward<T, FWD_PEN_NL, le>
#define K_FWD_PLIN(le) k_row_forward<T, FWD_PEN_LIN, le>
#define K_INVP(le) k_row_inverse<T, le, (kF32<T> ? INV_UV : INV_PSI)>
#define K_INVR(le) k_row_inverse<T, le, (kF32<T> ? INV_WUV : INV_WP)>
#define K_INVPSI(le) k_row_inverse<T, le, INV_PSI>
#define K_COLP(le) k_col_poisson<T, le, kF32<T>>
#define K_COLPSI(le) k_col_poisson<T, le, false>
#define K_COLU(le) k_col_update<T, le>

class RaggedF32;

template <class T>
class StepperImpl : public StepperBase {
    friend class RaggedF32;   // drives float steppers' data through the ragged launches

  public:
    using C = Cx<T>;
    StepperImpl(const nsstab_config& cfg, int nsets, const double* Re, const double* D, int per_set,
                cudaStream_t s)
        : cfg_(cfg), stream_(s), S_(nsets), bper_(per_set), B_(nsets * per_set) {
        for (int k = 0; k < nsets; ++k) {
            Re_.push_back(Re ? Re[k] : cfg.Re);
            D_.push_back(D ? D[k] : cfg.cyl_D);
        }
    }
    ~StepperImpl() override { release(); }

    int init() override;
    int members() const override { return B_; }
    int sets() const override { return S_; }
    int poisson(const double* omega, double* psi) override;
    int step_nonlinear(double* omega, int nsteps) override;
    int set_base(const double* base_omega) override;
    int set_base_ptrs(const double* const* base_omegas) override;
    int step_linear(const double* v_in, double* v_out, int nsteps) override;
    int step_linear_ptrs(const double* const* in, double* const* out, int nsteps) override;
    int tangent(const double* q, const double* v_in, double* v_out, int nsteps) override;
    int residual(const double* q, double* r) override;
    int sfd(double* omega, double chi, double Delta, double tol, long max_steps, int check_every,
            double* r, long* steps) override;
    int launches_per_step() const override { return rollR_ ? 4 : kNumStepKernels; }
    int profile_linear(const double* v, int nsteps, double* ms) override;
    int autotune(int reps, int* chosen) override;
    int plan_of(int kid, int* le, int* per) const override {
        if (kid < 0 || kid >= kNumStepKernels) return NSSTAB_ERR_INVALID_ARG;
        *le = plan_[kid].le;
        *per = plan_[kid].per;
        return NSSTAB_OK;
    }
    int set_plan(int kid, int le, int per) override;
    int set_fused_rows(int R) override;
    int fused_rows() const override { return rollR_; }

  private:
    nsstab_config cfg_;
    cudaStream_t stream_;
    int S_, bper_, B_;
    std::vector<double> Re_, D_;
    cudaStream_t cap_ = nullptr;   // private stream used only to capture graphs
    Fields<T> f_{};
    int nx_ = 0, ny_ = 0, nxh_ = 0;
    size_t n_ = 0, nc_ = 0;
    std::vector<void*> allocs_;
    T* Wsave_ = nullptr;
    C* Nhsave_ = nullptr;
    double* red_ = nullptr;          // device partials [B][kRedBlocks]
    double* red_host_ = nullptr;     // pinned
    unsigned char* active_ = nullptr;
    unsigned char* tmask_ = nullptr;               // device {1, 0, 0, 1}: member 0 alone, member 1 alone
    const unsigned char* act_override_ = nullptr;  // mask for the next launches (null: the stepper's own)
    bool xn_x4_ = false;                           // k_col_update reads N from X4 (fused row passes)
    std::vector<unsigned char> active_host_;
    const double** ptr_in_ = nullptr;   // device arrays of B member pointers
    double** ptr_out_ = nullptr;
    std::vector<const double*> pin_host_;
    std::vector<double*> pout_host_;
    bool have_base_ = false;
    Launch plan_[kNumStepKernels];
    int rollR_ = 0;                // fused FP32 row passes over strips of rollR_ rows (0: six-kernel step)
    RollShape rs_{};
    T scale_ = T(1);
    struct GraphKey {
        int nsteps, flags;
        bool operator<(const GraphKey& o) const { return nsteps != o.nsteps ? nsteps < o.nsteps : flags < o.flags; }
    };
    std::map<GraphKey, cudaGraphExec_t> graphs_;

    template <class P> int dalloc(P** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(P));
        if (e != cudaSuccess) {
            set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? NSSTAB_ERR_OUT_OF_MEMORY : NSSTAB_ERR_CUDA;
        }
        allocs_.push_back(q);
        *p = static_cast<P*>(q);
        return NSSTAB_OK;
    }
    void clear_graphs() {
        for (auto& kv : graphs_) cudaGraphExecDestroy(kv.second);
        graphs_.clear();
    }
    void release() {
        cudaStreamSynchronize(stream_);
        clear_graphs();
        if (cap_) cudaStreamDestroy(cap_);
        cap_ = nullptr;
        for (void* p : allocs_) cudaFree(p);
        allocs_.clear();
        if (red_host_) cudaFreeHost(red_host_);
        red_host_ = nullptr;
    }
    int build_tables();
    Launch make_plan(int kid, int le, int per, int tm = 1) const;
    Launch with_tm2(int kid, const Launch& L) const;
    int set_plan_tm(int kid, int le, int per, int tm);
    Launch default_plan(int kid) const;
    int set_smem_attr(int kid, const Launch& L);

    int set_active(const std::vector<unsigned char>& a);
    int all_active() { return set_active(std::vector<unsigned char>(B_, 1)); }
    int gather(const double* const* src);                // W[m] <- src[m] (null: skip)
    int scatter(const T* from, double* const* dst);      // dst[m] <- from[m] (null: skip)
    int gather_contig(const double* src, int count);     // members 0..count-1 from [count][n]
    int scatter_contig(const T* from, double* dst);      // all members to [B][n]
    int launch(int kid, cudaStream_t st, bool linear, bool sfd, bool do_fft, bool first);
    int launch_roll(bool pen, cudaStream_t st, bool linear, bool sfd, bool do_fft, bool write_w);
    RollShape roll_shape(int R) const;
    int launch_plain(cudaStream_t st);
    int transform_W();                                   // X1 = x-spectrum of W
    int stream_function(cudaStream_t st);                // Wh, X2 (X3), P (U, V) from X1
    int psi_function(cudaStream_t st);                   // Wh, X2, P from X1
    int issue_steps(cudaStream_t st, int nsteps, bool linear, bool sfd, bool first_ab1, bool fft_last,
                    bool tangent = false);
    int run_steps(int nsteps, bool linear, bool sfd, bool fft_last, bool first_ab1 = true, bool tangent = false);
    int alloc_base_fields();
    int sumsq_diff(const T* a, const T* b, double* out);   // out[B]
    int time_kernel(int kid, const Launch& L, int reps, float* ms);
};

// ---------------------------------------------------------- launch plans

// Transforms per member of launch kid: row pairs or rows for the row passes
// (see InvIO), columns for the column passes.
template <class T> static int seq_count(int kid, int nx, int ny) {
    switch (kid) {
        case KCOLP:
        case KCOLU: return nx / 2;
        case KINVP: return kF32<T> ? ny : ny / 2;
        case KINVR: return kF32<T> ? ny + ny / 2 : ny;
        default: return ny / 2;
    }
}

// Column passes with two or more inverse transforms per column (col_update;
// col_poisson of the FP32 stepper) may run blocks of twice the threads of
// one transform round (tm = 2): the inverse transforms then proceed side by
// side, and twice the loads are in flight.
template <class T> static bool tm2_allowed(int kid) { return kid == KCOLU || (kid == KCOLP && kF32<T>); }

template <class T> Launch StepperImpl<T>::make_plan(int kid, int le, int per, int tm) const {
    Launch L;
    if (tm != 1 && !(tm == 2 && tm2_allowed<T>(kid))) return L;
    const bool row = (kid == KINVP || kid == KFWDR || kid == KINVR || kid == KFWDP);
    const int N = row ? nx_ : ny_;
    const int logN = row ? ilog2(nx_) : ilog2(ny_);
    const int count = seq_count<T>(kid, nx_, ny_);
    // shared-memory sequences per unit
    const int nseq_smem = (kid == KCOLU) ? 3 : (kid == KCOLP && kF32<T>) ? 2 : 1;
    if (le < 1 || le > 3 || logN < le || per < 1 || !is_pow2(per) || per > count) return L;
    if (kF32<T> && kid == KINVR && per > ny_ / 2) return L;   // blocks must not straddle the two parts
    const int threads = per * (N >> le) * tm;
    const int rp = row ? per : ((N >> le) < 32 ? 32 / (N >> le) : 1);
    const size_t smem = (size_t)per * nseq_smem * seq_stride(N, rp, (int)sizeof(C) / 4) * sizeof(C);
    if (threads > 1024 || smem > kMaxSmem) return L;
    L.per = per;
    L.logper = ilog2(per);
    L.le = le;
    L.tm = tm;
    L.blocks = count / per;
    L.threads = threads;
    L.smem = smem;
    L.ok = true;
    return L;
}

// Default: the largest elements-per-thread (fewest FP64 operations per
// point) that still gives every SM sub-partition a warp over the whole
// batch, then enough sequences per block for at least two warps.
template <class T> Launch StepperImpl<T>::default_plan(int kid) const {
    const bool row = (kid == KINVP || kid == KFWDR || kid == KINVR || kid == KFWDP);
    const int N = row ? nx_ : ny_;
    const long count = seq_count<T>(kid, nx_, ny_);
    const long target = 4L * 152 * 32;   // one warp per SM sub-partition
    int le = 3;
    while (le > 2 && (long)B_ * count * (N >> le) < target) --le;
    if (ilog2(N) < le) le = ilog2(N);
    int per = 1;
    while (per * (N >> le) < 64 && 2 * per <= count) per *= 2;
    Launch L = make_plan(kid, le, per);
    while ((!L.ok || L.threads > max_threads_for<T>(kid, le)) && per > 1) L = make_plan(kid, le, per /= 2);
    while ((!L.ok || L.threads > max_threads_for<T>(kid, le)) && le > 1) L = make_plan(kid, --le, 1);
    return with_tm2(kid, L);
}

// The same plan with tm = 2 where the kernel allows it, the block fits, and
// the grid is short of warps (fewer than 8 per SM at tm = 1 over the whole
// batch): doubling the block pays for latency-bound small grids, while on
// large grids it only raises the register pressure.
template <class T> Launch StepperImpl<T>::with_tm2(int kid, const Launch& L) const {
    if (!L.ok || !tm2_allowed<T>(kid)) return L;
    if ((long)B_ * L.blocks * L.threads >= 8L * 152 * 32) return L;
    const Launch L2 = make_plan(kid, L.le, L.per, 2);
    return (L2.ok && L2.threads <= max_threads_for<T>(kid, L.le)) ? L2 : L;
}

// The dynamic shared-memory limit is an attribute of the kernel function,
// shared by every stepper in the process: each one raises it to the same
// library-wide cap (never to its own plan's size), so steppers on other
// grids running concurrently in other threads can never lower it below
// what their launches need.  A launch still requests only L.smem.
template <class T> int StepperImpl<T>::set_smem_attr(int kid, const Launch& L) {
    if (L.smem > kMaxSmem) {
        set_error("launch plan needs more shared memory than the library allows");
        return NSSTAB_ERR_INVALID_ARG;
    }
    const int sm = (int)kMaxSmem;
#define NS_ATTR(fn) NS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))
#define NS_ATTR_LE(KERNEL)                 \
    switch (L.le) {                        \
        case 1: NS_ATTR(KERNEL(1)); break; \
        case 2: NS_ATTR(KERNEL(2)); break; \
        default: NS_ATTR(KERNEL(3)); break; \
    }
    switch (kid) {
        case KCOLP: NS_ATTR_LE(K_COLP); NS_ATTR_LE(K_COLPSI); break;
        case KINVP: NS_ATTR_LE(K_INVP); NS_ATTR_LE(K_INVPSI); break;
        case KINVR: NS_ATTR_LE(K_INVR); break;
        case KFWDR: NS_ATTR_LE(K_FWD_RNL); NS_ATTR_LE(K_FWD_RLIN); NS_ATTR_LE(K_FWD_PLAIN); break;
        case KCOLU: NS_ATTR_LE(K_COLU); break;
        default: NS_ATTR_LE(K_FWD_PNL); NS_ATTR_LE(K_FWD_PLIN); break;
    }
    return NSSTAB_OK;
}

// Largest block the register budget of the kernel instantiations behind
// launch `kid` with 2^le elements per thread allows.
template <class T> int max_threads_for(int kid, int le) {
    cudaFuncAttributes a;
    int m = 1024;
    auto take = [&](const void* fn) {
        if (cudaFuncGetAttributes(&a, fn) == cudaSuccess) m = std::min(m, a.maxThreadsPerBlock);
        else m = 0;
    };
#define NS_TAKE_LE(KERNEL)                            \
    switch (le) {                                     \
        case 1: take((const void*)KERNEL(1)); break;  \
        case 2: take((const void*)KERNEL(2)); break;  \
        default: take((const void*)KERNEL(3)); break; \
    }
    switch (kid) {
        case KCOLP: NS_TAKE_LE(K_COLP); NS_TAKE_LE(K_COLPSI); break;
        case KINVP: NS_TAKE_LE(K_INVP); NS_TAKE_LE(K_INVPSI); break;
        case KINVR: NS_TAKE_LE(K_INVR); break;
        case KFWDR: NS_TAKE_LE(K_FWD_RNL); NS_TAKE_LE(K_FWD_RLIN); NS_TAKE_LE(K_FWD_PLAIN); break;
        case KCOLU: NS_TAKE_LE(K_COLU); break;
        default: NS_TAKE_LE(K_FWD_PNL); NS_TAKE_LE(K_FWD_PLIN); break;
    }
    return m;
}

template <class T> int StepperImpl<T>::set_plan(int kid, int le, int per) {
    if (kid < 0 || kid >= kNumStepKernels) {
        set_error("set_plan: bad kernel id");
        return NSSTAB_ERR_INVALID_ARG;
    }
    return set_plan_tm(kid, le, per, with_tm2(kid, make_plan(kid, le, per)).tm);
}

template <class T> int StepperImpl<T>::set_plan_tm(int kid, int le, int per, int tm) {
    const Launch L = make_plan(kid, le, per, tm);
    if (!L.ok || L.threads > max_threads_for<T>(kid, le)) {
        set_error("set_plan: configuration not valid for this grid");
        return NSSTAB_ERR_INVALID_ARG;
    }
    NS_TRY(set_smem_attr(kid, L));
    plan_[kid] = L;
    clear_graphs();
    return NSSTAB_OK;
}

#define NS_DISPATCH_LE(L, CALL)  \
    switch ((L).le) {            \
        case 1: CALL(1); break;  \
        case 2: CALL(2); break;  \
        default: CALL(3); break; \
    }

template <class T> int StepperImpl<T>::launch_plain(cudaStream_t st) {
    const Launch& L = plan_[KFWDR];
    const dim3 g(L.blocks, B_);
#define CALL_PLAIN(le) k_row_forward<T, FWD_PLAIN, le><<<g, L.threads, L.smem, st>>>(f_, L.per, L.logper, false, true)
    NS_DISPATCH_LE(L, CALL_PLAIN);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::launch(int kid, cudaStream_t st, bool linear, bool sfd, bool do_fft, bool first) {
    const Launch& L = plan_[kid];
    const dim3 g(L.blocks, B_);
    Fields<T> fl = f_;   // passed by value: a graph capture records this launch's mask
    if (act_override_) fl.active = act_override_;
    switch (kid) {
        case KCOLP: {
#define CALL_COLP(le) k_col_poisson<T, le, kF32<T>><<<g, L.threads, L.smem, st>>>(fl, L.per, scale_)
            NS_DISPATCH_LE(L, CALL_COLP);
            break;
        }
        case KINVP: {
#define CALL_INVP(le) K_INVP(le)<<<g, L.threads, L.smem, st>>>(fl, L.per, L.logper)
            NS_DISPATCH_LE(L, CALL_INVP);
            break;
        }
        case KFWDR: {
#define CALL_FRL(le) k_row_forward<T, FWD_RHS_LIN, le><<<g, L.threads, L.smem, st>>>(fl, L.per, L.logper, false, true)
#define CALL_FRN(le) k_row_forward<T, FWD_RHS_NL, le><<<g, L.threads, L.smem, st>>>(fl, L.per, L.logper, false, true)
            if (linear) {
                NS_DISPATCH_LE(L, CALL_FRL);
            } else {
                NS_DISPATCH_LE(L, CALL_FRN);
            }
            break;
        }
        case KCOLU: {
            if (xn_x4_) fl.XN = f_.X4;
            const T c1 = first ? T(1) : T(1.5), c0 = first ? T(0) : T(-0.5);
#define CALL_COLU(le) k_col_update<T, le><<<g, L.threads, L.smem, st>>>(fl, L.per, c1, c0, first)
            NS_DISPATCH_LE(L, CALL_COLU);
            break;
        }
        case KINVR: {
#define CALL_INVR(le) K_INVR(le)<<<g, L.threads, L.smem, st>>>(fl, L.per, L.logper)
            NS_DISPATCH_LE(L, CALL_INVR);
            break;
        }
        default: {
#define CALL_FPL(le) k_row_forward<T, FWD_PEN_LIN, le><<<g, L.threads, L.smem, st>>>(fl, L.per, L.logper, sfd, do_fft)
#define CALL_FPN(le) k_row_forward<T, FWD_PEN_NL, le><<<g, L.threads, L.smem, st>>>(fl, L.per, L.logper, sfd, do_fft)
            if (linear) {
                NS_DISPATCH_LE(L, CALL_FPL);
            } else {
                NS_DISPATCH_LE(L, CALL_FPN);
            }
            break;
        }
    }
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

// Shape of the fused row passes for strips of R rows (nunits = 0: the grid
// or arithmetic does not allow it).
template <class T> RollShape StepperImpl<T>::roll_shape(int R) const {
    RollShape r{};
    if (!kF32<T> || nx_ < 64 || nx_ > kRollPoints || R < 2 || (R & 1) || R > ny_ || ny_ % R != 0) return r;
    r.R = R;
    r.G = std::min(kRollPoints / nx_, ny_ / R);
    r.upm = ny_ / (R * r.G);
    r.nunits = B_ * r.upm;
    return r;
}

template <class T> int StepperImpl<T>::set_fused_rows(int R) {
    if (R == 0) {
        rollR_ = 0;
        clear_graphs();
        return NSSTAB_OK;
    }
    const RollShape r = roll_shape(R);
    if (r.nunits == 0) {
        set_error("fused row passes need the FP32 stepper, 64 <= nx <= 2048 and an even R dividing ny");
        return NSSTAB_ERR_INVALID_ARG;
    }
    if constexpr (kF32<T>) {
        const int sm = (int)roll_smem(kRollPoints);
        NS_CUDA(cudaFuncSetAttribute(k_row_roll<FWD_RHS_NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        NS_CUDA(cudaFuncSetAttribute(k_row_roll<FWD_RHS_LIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        NS_CUDA(cudaFuncSetAttribute(k_row_roll<FWD_PEN_NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        NS_CUDA(cudaFuncSetAttribute(k_row_roll<FWD_PEN_LIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    }
    rollR_ = R;
    rs_ = r;
    clear_graphs();
    return NSSTAB_OK;
}

// One fused row pass over every active member: persistent blocks, one per
// SM at most (the pass holds 96 G nx bytes of shared memory).
template <class T>
int StepperImpl<T>::launch_roll(bool pen, cudaStream_t st, bool linear, bool sfd, bool do_fft, bool write_w) {
    if constexpr (kF32<T>) {
        RollShape r = rs_;
        r.write_w = write_w ? 1 : 0;
        r.do_fft = do_fft ? 1 : 0;
        Fields<T> fl = f_;
        if (act_override_) fl.active = act_override_;
        const int blocks = std::min(r.nunits, 152);
        const size_t smem = roll_smem(r.G * nx_) ;
        if (!pen) {
            if (linear) k_row_roll<FWD_RHS_LIN><<<blocks, kRollThreads, smem, st>>>(fl, r, false);
            else k_row_roll<FWD_RHS_NL><<<blocks, kRollThreads, smem, st>>>(fl, r, false);
        } else {
            if (linear) k_row_roll<FWD_PEN_LIN><<<blocks, kRollThreads, smem, st>>>(fl, r, sfd);
            else k_row_roll<FWD_PEN_NL><<<blocks, kRollThreads, smem, st>>>(fl, r, sfd);
        }
        NS_LAUNCH_CHECK();
        return NSSTAB_OK;
    } else {
        set_error("fused row passes exist for the FP32 stepper only");
        return NSSTAB_ERR_INVALID_ARG;
    }
}

// --------------------------------------------------------------- tables

template <class T> int StepperImpl<T>::build_tables() {
    const int nx = nx_, ny = ny_, nxh = nxh_;
    const double dx = cfg_.Lx / nx, dy = cfg_.Ly / ny;
    const double dt = cfg_.dt;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    // per-pass twiddle tables (see fft.cuh) in extended precision, rounded once
    auto build_tw = [&](int N, int LE, std::vector<C>& out) {
        const int logN = ilog2(N);
        out.clear();
        int nsl = 0, rem = logN;
        auto pass = [&](int LR) {
            const int Ns = 1 << nsl, R = 1 << LR;
            for (int r = 0; r < R; ++r)
                for (int k = 0; k < Ns; ++k) {
                    const long double a = two_pi * (long double)(r * k) / (long double)(Ns * R);
                    const long double c = cosl(a), sn = -sinl(a);
                    const T ch = (T)(double)c, sh = (T)(double)sn;
                    out.push_back(mk<T>(ch, sh));
                    if (kTwWidth<T> == 2)   // FP32: the rounding errors of hi, next to it
                        out.push_back(mk<T>((T)(double)(c - (long double)(double)ch),
                                            (T)(double)(sn - (long double)(double)sh)));
                }
            nsl += LR;
            rem -= LR;
        };
        while (rem >= LE) pass(LE);
        if (rem > 0) pass(rem);
    };
    // spectral operators over kx in [0, nx/2], ky in [0, ny): eigenvalue of
    // the periodic 5-point Laplacian lam = lx(kx) + ly(ky); tA, tB per set
    const size_t nt = (size_t)(nxh + 1) * ny;
    std::vector<T> tA(nt * S_), tB(nt * S_), tP(nt);
    const double scale = 1.0 / ((double)nx * (double)ny);
    for (int kx = 0; kx <= nxh; ++kx) {
        const double sx = std::sin(kPi * kx / nx);
        const double lx = -(4.0 / (dx * dx)) * sx * sx;
        for (int ky = 0; ky < ny; ++ky) {
            const double sy = std::sin(kPi * ky / ny);
            const double lam = lx - (4.0 / (dy * dy)) * sy * sy;
            const size_t g = (size_t)kx * ny + ky;
            tP[g] = (kx == 0 && ky == 0) ? T(0) : (T)(-1.0 / lam);
            for (int k = 0; k < S_; ++k) {
                const double nu = 1.0 / Re_[k];
                if (kx == 0 && ky == 0) {   // the mean mode is removed: A = B = 0
                    tA[k * nt + g] = kF32<T> ? (T)(-scale) : T(0);
                    tB[k * nt + g] = T(0);
                    continue;
                }
                const double a = 1.0 + 0.5 * nu * dt * lam;
                const double b = 1.0 - 0.5 * nu * dt * lam;
                // FP32: A - 1 = nu dt lam / b, formed without cancellation
                tA[k * nt + g] = kF32<T> ? (T)(scale * (nu * dt * lam) / b) : (T)(scale * a / b);
                tB[k * nt + g] = (T)(scale * dt / b);
            }
        }
    }
    // penalisation coefficients from the cylinder mask and the fringe, per set
    std::vector<T> cS(n_ * S_), cG(n_ * S_);
    const double w = 0.5 * cfg_.mask_cells * dx;
    const double xs = (1.0 - cfg_.sponge_frac) * cfg_.Lx;
    for (int k = 0; k < S_; ++k) {
        const double Dk = D_[k], R = 0.5 * Dk;
        for (int j = 0; j < ny; ++j) {
            const double y = j * dy;
            for (int i = 0; i < nx; ++i) {
                const double x = i * dx;
                double chi = 0.0;
                if (Dk > 0.0) {
                    double ddx = std::fmod(x - cfg_.cyl_x + 0.5 * cfg_.Lx, cfg_.Lx);
                    if (ddx < 0) ddx += cfg_.Lx;
                    ddx -= 0.5 * cfg_.Lx;
                    double ddy = std::fmod(y - cfg_.cyl_y + 0.5 * cfg_.Ly, cfg_.Ly);
                    if (ddy < 0) ddy += cfg_.Ly;
                    ddy -= 0.5 * cfg_.Ly;
                    const double r = std::sqrt(ddx * ddx + ddy * ddy);
                    if (r <= R - w) chi = 1.0;
                    else if (r >= R + w) chi = 0.0;
                    else chi = 0.5 * (1.0 - std::sin(kPi * (r - R) / (2.0 * w)));
                }
                double sig = 0.0;
                if (cfg_.sponge_sigma > 0.0 && cfg_.sponge_frac > 0.0 && x >= xs) {
                    const double sn = std::sin(kPi * (x - xs) / (cfg_.sponge_frac * cfg_.Lx));
                    sig = cfg_.sponge_sigma * sn * sn;
                }
                const double s = dt * (chi / cfg_.eta + sig);
                const size_t c = k * n_ + (size_t)j * nx + i;
                cS[c] = (T)(s / (1.0 + s));
                cG[c] = (T)(dt * sig * cfg_.Uinf / (1.0 + s));
            }
        }
    }
    for (int le = 1; le <= 3; ++le) {
        std::vector<C> tx, ty;
        if (ilog2(nx) >= le) {
            build_tw(nx, le, tx);
            NS_CUDA(cudaMemcpy((void*)f_.twx[le], tx.data(), tx.size() * sizeof(C), cudaMemcpyHostToDevice));
        }
        if (ilog2(ny) >= le) {
            build_tw(ny, le, ty);
            NS_CUDA(cudaMemcpy((void*)f_.twy[le], ty.data(), ty.size() * sizeof(C), cudaMemcpyHostToDevice));
        }
    }
    NS_CUDA(cudaMemcpyAsync((void*)f_.tA, tA.data(), tA.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
    NS_CUDA(cudaMemcpyAsync((void*)f_.tB, tB.data(), tB.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
    NS_CUDA(cudaMemcpyAsync((void*)f_.tP, tP.data(), tP.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
    // centred-difference symbols: D_x <-> i sin(2 pi kx/nx)/dx, D_y alike
    std::vector<T> tDx(nxh + 1), tDy(ny);
    for (int kx = 0; kx <= nxh; ++kx) tDx[kx] = (kx == 0 || kx == nxh) ? T(0) : (T)(std::sin(2.0 * kPi * kx / nx) / dx);
    for (int ky = 0; ky < ny; ++ky) tDy[ky] = (2 * ky == ny || ky == 0) ? T(0) : (T)(std::sin(2.0 * kPi * ky / ny) / dy);
    if (f_.tDx) {
        NS_CUDA(cudaMemcpyAsync((void*)f_.tDx, tDx.data(), tDx.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
        NS_CUDA(cudaMemcpyAsync((void*)f_.tDy, tDy.data(), tDy.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
    }
    NS_CUDA(cudaMemcpyAsync((void*)f_.cS, cS.data(), cS.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
    NS_CUDA(cudaMemcpyAsync((void*)f_.cG, cG.data(), cG.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
    NS_CUDA(cudaStreamSynchronize(stream_));   // host vectors go out of scope
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::init() {
    nx_ = cfg_.nx;
    ny_ = cfg_.ny;
    nxh_ = nx_ / 2;
    n_ = (size_t)nx_ * ny_;
    nc_ = (size_t)nxh_ * ny_;
    const size_t nt = (size_t)(nxh_ + 1) * ny_;
    f_.nx = nx_;
    f_.ny = ny_;
    f_.nxh = nxh_;
    f_.logx = ilog2(nx_);
    f_.logy = ilog2(ny_);
    f_.bper = bper_;
    f_.fs = n_;
    f_.cs = nc_;
    f_.ts = nt;
    f_.idx2 = (T)(1.0 / (2.0 * cfg_.Lx / nx_));
    f_.idy2 = (T)(1.0 / (2.0 * cfg_.Ly / ny_));
    f_.Uinf = (T)cfg_.Uinf;
    scale_ = (T)(1.0 / ((double)nx_ * (double)ny_));
    f_.scale = scale_;
    const size_t B = B_, S = S_;
    T *W, *P, *cS, *cG, *tA, *tB, *tP;
    C *X1, *X2, *Wh, *Nh;
    NS_TRY(dalloc(&W, B * n_));
    NS_TRY(dalloc(&P, B * n_));
    NS_TRY(dalloc(&X1, B * nc_));
    NS_TRY(dalloc(&X2, B * nc_));
    NS_TRY(dalloc(&Wh, B * nc_));
    NS_TRY(dalloc(&Nh, B * nc_));
    NS_TRY(dalloc(&cS, S * n_));
    NS_TRY(dalloc(&cG, S * n_));
    NS_TRY(dalloc(&tA, S * nt));
    NS_TRY(dalloc(&tB, S * nt));
    NS_TRY(dalloc(&tP, nt));
    if (kF32<T>) {
        T *U, *V, *tDx, *tDy;
        C* X3;
        NS_TRY(dalloc(&U, B * n_));
        NS_TRY(dalloc(&V, B * n_));
        NS_TRY(dalloc(&X3, B * nc_));
        C* X4;
        NS_TRY(dalloc(&X4, B * nc_));
        f_.X4 = X4;
        NS_CUDA(cudaMemsetAsync(X4, 0, B * nc_ * sizeof(C), stream_));
        NS_TRY(dalloc(&tDx, (size_t)nxh_ + 1));
        NS_TRY(dalloc(&tDy, (size_t)ny_));
        f_.U = U; f_.V = V; f_.X3 = X3; f_.tDx = tDx; f_.tDy = tDy;
        NS_CUDA(cudaMemsetAsync(U, 0, B * n_ * sizeof(T), stream_));
        NS_CUDA(cudaMemsetAsync(V, 0, B * n_ * sizeof(T), stream_));
        NS_CUDA(cudaMemsetAsync(X3, 0, B * nc_ * sizeof(C), stream_));
    }
    for (int le = 1; le <= 3; ++le) {
        C *tx, *ty;
        NS_TRY(dalloc(&tx, (size_t)2 * kTwWidth<T> * nx_));
        NS_TRY(dalloc(&ty, (size_t)2 * kTwWidth<T> * ny_));
        f_.twx[le] = tx;
        f_.twy[le] = ty;
    }
    f_.twx[0] = f_.twx[1];
    f_.twy[0] = f_.twy[1];
    NS_TRY(dalloc(&red_, B * kRedBlocks));
    NS_TRY(dalloc(&active_, B));
    NS_TRY(dalloc(&ptr_in_, B));
    NS_TRY(dalloc(&ptr_out_, B));
    NS_CUDA(cudaMallocHost((void**)&red_host_, B * kRedBlocks * sizeof(double)));
    f_.W = W; f_.P = P; f_.cS = cS; f_.cG = cG;
    f_.X1 = X1; f_.X2 = X2; f_.Wh = Wh; f_.Nh = Nh;
    f_.XN = X1;
    f_.tA = tA; f_.tB = tB; f_.tP = tP;
    f_.Y = nullptr;
    f_.Ub = f_.Vb = f_.DxOb = f_.DyOb = nullptr;
    f_.active = active_;
    NS_TRY(build_tables());
    // zero the workspace so that timing runs of the autotuner see finite data
    NS_CUDA(cudaMemsetAsync(f_.W, 0, B * n_ * sizeof(T), stream_));
    NS_CUDA(cudaMemsetAsync(f_.P, 0, B * n_ * sizeof(T), stream_));
    NS_CUDA(cudaMemsetAsync(f_.X1, 0, B * nc_ * sizeof(C), stream_));
    NS_CUDA(cudaMemsetAsync(f_.X2, 0, B * nc_ * sizeof(C), stream_));
    NS_CUDA(cudaMemsetAsync(f_.Wh, 0, B * nc_ * sizeof(C), stream_));
    NS_CUDA(cudaMemsetAsync(f_.Nh, 0, B * nc_ * sizeof(C), stream_));
    NS_TRY(all_active());
    NS_CUDA(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
    for (int k = 0; k < kNumStepKernels; ++k) {
        const Launch L = default_plan(k);
        if (!L.ok) {
            set_error("grid too large for the shared-memory FFT");
            return NSSTAB_ERR_INVALID_ARG;
        }
        NS_TRY(set_plan_tm(k, L.le, L.per, L.tm));
    }

    NS_CUDA(cudaStreamSynchronize(stream_));
    return NSSTAB_OK;
}

// ------------------------------------------------- member data movement

// Host vectors are pageable: cudaMemcpyAsync stages them before returning,
// so they may be reused by the next call at once.
template <class T> int StepperImpl<T>::set_active(const std::vector<unsigned char>& a) {
    active_host_ = a;
    NS_CUDA(cudaMemcpyAsync(active_, active_host_.data(), B_, cudaMemcpyHostToDevice, stream_));
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::gather(const double* const* src) {
    pin_host_.assign(src, src + B_);
    NS_CUDA(cudaMemcpyAsync(ptr_in_, pin_host_.data(), B_ * sizeof(double*), cudaMemcpyHostToDevice, stream_));
    k_gather<T><<<dim3(kPtBlocks, B_), 256, 0, stream_>>>(ptr_in_, f_.W, n_, n_);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::scatter(const T* from, double* const* dst) {
    pout_host_.assign(dst, dst + B_);
    NS_CUDA(cudaMemcpyAsync(ptr_out_, pout_host_.data(), B_ * sizeof(double*), cudaMemcpyHostToDevice, stream_));
    k_scatter<T><<<dim3(kPtBlocks, B_), 256, 0, stream_>>>(from, ptr_out_, n_, n_);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::gather_contig(const double* src, int count) {
    std::vector<const double*> p(B_, nullptr);
    for (int m = 0; m < count; ++m) p[m] = src + (size_t)m * n_;
    return gather(p.data());
}

template <class T> int StepperImpl<T>::scatter_contig(const T* from, double* dst) {
    std::vector<double*> p(B_);
    for (int m = 0; m < B_; ++m) p[m] = dst + (size_t)m * n_;
    return scatter(from, p.data());
}

// ------------------------------------------------------------- stepping

template <class T> int StepperImpl<T>::transform_W() { return launch_plain(stream_); }

template <class T> int StepperImpl<T>::stream_function(cudaStream_t st) {
    NS_TRY(launch(KCOLP, st, false, false, true, false));
    return launch(KINVP, st, false, false, true, false);
}

// P = psi from X1 for every stepper (kVel steppers carry u', v in the step
// and form psi only here): the psi variant of the column pass, then the
// row pairs of X2, with the launch shapes of KCOLP and KINVP.
template <class T> int StepperImpl<T>::psi_function(cudaStream_t st) {
    if (!kF32<T>) return stream_function(st);
    const Launch& Lc = plan_[KCOLP];
    const dim3 gc(Lc.blocks, B_);
#define CALL_COLPSI(le) k_col_poisson<T, le, false><<<gc, Lc.threads, Lc.smem, st>>>(f_, Lc.per, scale_)
    NS_DISPATCH_LE(Lc, CALL_COLPSI);
    NS_LAUNCH_CHECK();
    Launch L = plan_[KINVP];   // ny rows -> ny/2 row pairs, each block at most as large
    while (L.per > ny_ / 2) L.per /= 2;
    L.logper = ilog2(L.per);
    L.blocks = (ny_ / 2) / L.per;
    L.threads = L.per * (nx_ >> L.le);
    L.smem = (size_t)L.per * seq_stride(nx_, L.per, (int)sizeof(C) / 4) * sizeof(C);
    const dim3 gr(L.blocks, B_);
#define CALL_INVPSI(le) K_INVPSI(le)<<<gr, L.threads, L.smem, st>>>(f_, L.per, L.logper)
    NS_DISPATCH_LE(L, CALL_INVPSI);
    NS_LAUNCH_CHECK();
    return NSSTAB_OK;
}

// Enqueue nsteps time steps on `st`.  first_ab1: the first of them is AB1.
// fft_last: the last step also forms the x-spectrum of its result.
template <class T>
int StepperImpl<T>::issue_steps(cudaStream_t st, int nsteps, bool linear, bool sfd, bool first_ab1, bool fft_last,
                                bool tangent) {
    if (tangent) {
        // co-integration (members: 0 = trajectory, 1 = perturbation): both
        // streamfunctions, the base fields of the trajectory's current
        // state, then each row pass in its own mode; the column passes
        // are the same for both
        for (int s = 0; s < nsteps; ++s) {
            const bool first = first_ab1 && s == 0;
            const bool fft = fft_last || (s + 1 < nsteps);
            NS_TRY(stream_function(st));
            k_base_fields<T><<<dim3(kPtBlocks, 1), 256, 0, st>>>(f_, (T*)f_.Ub, (T*)f_.Vb, (T*)f_.DxOb,
                                                                 (T*)f_.DyOb);
            NS_LAUNCH_CHECK();
            act_override_ = tmask_;
            int rc = launch(KFWDR, st, false, false, true, first);
            act_override_ = tmask_ + 2;
            if (rc == NSSTAB_OK) rc = launch(KFWDR, st, true, false, true, first);
            act_override_ = nullptr;
            NS_TRY(rc);
            NS_TRY(launch(KCOLU, st, true, false, true, first));
            NS_TRY(launch(KINVR, st, true, false, true, first));
            act_override_ = tmask_;
            rc = launch(KFWDP, st, false, false, fft, first);
            act_override_ = tmask_ + 2;
            if (rc == NSSTAB_OK) rc = launch(KFWDP, st, true, false, fft, first);
            act_override_ = nullptr;
            NS_TRY(rc);
        }
        return NSSTAB_OK;
    }
    if (rollR_) {
        // four kernels: column Poisson pass, fused RHS row pass, column
        // update, fused penalisation row pass (omega to W on the last step)
        for (int s = 0; s < nsteps; ++s) {
            const bool first = first_ab1 && s == 0;
            NS_TRY(launch(KCOLP, st, false, false, true, first));
            NS_TRY(launch_roll(false, st, linear, false, true, false));
            xn_x4_ = true;
            const int rc = launch(KCOLU, st, linear, false, true, first);
            xn_x4_ = false;
            NS_TRY(rc);
            NS_TRY(launch_roll(true, st, linear, sfd, fft_last || (s + 1 < nsteps), s + 1 == nsteps));
        }
        return NSSTAB_OK;
    }
    for (int s = 0; s < nsteps; ++s) {
        const bool first = first_ab1 && s == 0;
        NS_TRY(stream_function(st));
        NS_TRY(launch(KFWDR, st, linear, false, true, first));
        NS_TRY(launch(KCOLU, st, linear, false, true, first));
        NS_TRY(launch(KINVR, st, linear, false, true, first));
        NS_TRY(launch(KFWDP, st, linear, sfd, fft_last || (s + 1 < nsteps), first));
    }
    return NSSTAB_OK;
}

// Run nsteps steps on the stepper's stream.  Long runs replay CUDA graphs of
// up to kGraphChunk steps, captured once per (length, flags) on a private
// stream and launched into the stepper's stream; the AB2 history carries
// from one chunk to the next through the workspace.  The active-member mask
// is read from device memory at run time, so graphs serve any subset.
template <class T>
int StepperImpl<T>::run_steps(int nsteps, bool linear, bool sfd, bool fft_last, bool first_ab1, bool tangent) {
    if (linear && !have_base_) {
        set_error("linearised step requested before a base flow was set");
        return NSSTAB_ERR_INVALID_ARG;
    }
    if (nsteps < 4) return issue_steps(stream_, nsteps, linear, sfd, first_ab1, fft_last, tangent);
    int done = 0;
    while (done < nsteps) {
        const int len = std::min(kGraphChunk, nsteps - done);
        const bool first = first_ab1 && done == 0;
        const bool last_fft = (done + len < nsteps) || fft_last;
        const GraphKey key{len, (linear ? 1 : 0) | (sfd ? 2 : 0) | (first ? 4 : 0) | (last_fft ? 8 : 0) |
                                    (tangent ? 16 : 0)};
        auto it = graphs_.find(key);
        if (it == graphs_.end()) {
            cudaGraph_t g = nullptr;
            NS_CUDA(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
            const int rc = issue_steps(cap_, len, linear, sfd, first, last_fft, tangent);
            const cudaError_t ec = cudaStreamEndCapture(cap_, &g);
            if (rc != NSSTAB_OK) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            NS_CUDA(ec);
            cudaGraphExec_t ex = nullptr;
            const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            NS_CUDA(ei);
            it = graphs_.emplace(key, ex).first;
        }
        NS_CUDA(cudaGraphLaunch(it->second, stream_));
        done += len;
    }
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::time_kernel(int kid, const Launch& L, int reps, float* ms) {
    const Launch saved = plan_[kid];
    plan_[kid] = L;
    cudaEvent_t e0, e1;
    NS_CUDA(cudaEventCreate(&e0));
    NS_CUDA(cudaEventCreate(&e1));
    int rc = launch(kid, stream_, false, false, true, false);   // warm-up
    if (rc == NSSTAB_OK) {
        cudaEventRecord(e0, stream_);
        for (int r = 0; r < reps && rc == NSSTAB_OK; ++r) rc = launch(kid, stream_, false, false, true, false);
        cudaEventRecord(e1, stream_);
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess && rc == NSSTAB_OK) {
            set_error(std::string("autotune: ") + cudaGetErrorString(e));
            rc = NSSTAB_ERR_CUDA;
        }
        cudaEventElapsedTime(ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan_[kid] = saved;
    return rc;
}

// Measure every valid (elements per thread, sequences per block) pair of
// each kernel on this grid and batch and keep the fastest.  Clobbers the
// workspace (never the base flow).  chosen[2k], chosen[2k+1] = (le, per).
template <class T> int StepperImpl<T>::autotune(int reps, int* chosen) {
    NS_TRY(all_active());
    for (int kid = 0; kid < kNumStepKernels; ++kid) {
        Launch best = plan_[kid];
        float best_ms = 1e30f;
        for (int le = 1; le <= 3; ++le) {
            for (int per = 1; per <= 16; per *= 2) {
                for (int tm = 1; tm <= 2; ++tm) {
                    const Launch L = make_plan(kid, le, per, tm);
                    if (!L.ok || L.threads < 32 || L.threads > max_threads_for<T>(kid, le)) continue;
                    NS_TRY(set_smem_attr(kid, L));
                    float ms = 0.f;
                    NS_TRY(time_kernel(kid, L, reps, &ms));
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = L;
                    }
                }
            }
        }
        NS_TRY(set_plan_tm(kid, best.le, best.per, best.tm));
        if (chosen) {
            chosen[2 * kid] = best.le;
            chosen[2 * kid + 1] = best.per;
        }
    }
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::profile_linear(const double* v, int nsteps, double* ms) {
    if (!have_base_) {
        set_error("profile: no base flow set");
        return NSSTAB_ERR_INVALID_ARG;
    }
    cudaEvent_t ev[kNumStepKernels + 1];
    for (int k = 0; k <= kNumStepKernels; ++k) NS_CUDA(cudaEventCreate(&ev[k]));
    for (int k = 0; k < kNumStepKernels; ++k) ms[k] = 0.0;
    int rc = all_active();
    if (rc == NSSTAB_OK) rc = gather_contig(v, B_);
    if (rc == NSSTAB_OK) rc = transform_W();
    for (int s = 0; s < nsteps && rc == NSSTAB_OK; ++s) {
        const bool first = (s == 0);
        for (int k = 0; k < kNumStepKernels && rc == NSSTAB_OK; ++k) {
            cudaEventRecord(ev[k], stream_);
            if (!rollR_) rc = launch(k, stream_, true, false, true, first);
            else if (k == KCOLP) rc = launch(k, stream_, true, false, true, first);
            else if (k == KCOLU) {
                xn_x4_ = true;
                rc = launch(k, stream_, true, false, true, first);
                xn_x4_ = false;
            }
            else if (k == KFWDR) rc = launch_roll(false, stream_, true, false, true, false);
            else if (k == KFWDP) rc = launch_roll(true, stream_, true, false, true, s + 1 == nsteps);
        }
        cudaEventRecord(ev[kNumStepKernels], stream_);
        if (rc != NSSTAB_OK) break;
        const cudaError_t e = cudaEventSynchronize(ev[kNumStepKernels]);
        if (e != cudaSuccess) {
            set_error(std::string("profile: ") + cudaGetErrorString(e));
            rc = NSSTAB_ERR_CUDA;
            break;
        }
        for (int k = 0; k < kNumStepKernels; ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            ms[k] += t;
        }
    }
    for (int k = 0; k <= kNumStepKernels; ++k) cudaEventDestroy(ev[k]);
    return rc;
}

template <class T> int StepperImpl<T>::poisson(const double* omega, double* psi) {
    NS_TRY(all_active());
    NS_TRY(gather_contig(omega, B_));
    NS_TRY(transform_W());
    NS_TRY(psi_function(stream_));
    return scatter_contig(f_.P, psi);
}

template <class T> int StepperImpl<T>::step_nonlinear(double* omega, int nsteps) {
    NS_TRY(all_active());
    NS_TRY(gather_contig(omega, B_));
    if (nsteps > 0) {
        NS_TRY(transform_W());
        NS_TRY(run_steps(nsteps, false, false, false));
    }
    return scatter_contig(f_.W, omega);
}

template <class T> int StepperImpl<T>::set_base(const double* base_omega) {
    std::vector<const double*> p(S_);
    for (int k = 0; k < S_; ++k) p[k] = base_omega + (size_t)k * n_;
    return set_base_ptrs(p.data());
}

template <class T> int StepperImpl<T>::alloc_base_fields() {
    if (!f_.Ub) {
        T *Ub, *Vb, *DxOb, *DyOb;
        NS_TRY(dalloc(&Ub, (size_t)S_ * n_));
        NS_TRY(dalloc(&Vb, (size_t)S_ * n_));
        NS_TRY(dalloc(&DxOb, (size_t)S_ * n_));
        NS_TRY(dalloc(&DyOb, (size_t)S_ * n_));
        f_.Ub = Ub; f_.Vb = Vb; f_.DxOb = DxOb; f_.DyOb = DyOb;
        clear_graphs();   // captured kernels carry the field pointers by value
    }
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::set_base_ptrs(const double* const* base_omegas) {
    NS_TRY(alloc_base_fields());
    // the S base flows go through member slots 0..S-1
    std::vector<unsigned char> a(B_, 0);
    std::vector<const double*> src(B_, nullptr);
    for (int k = 0; k < S_; ++k) {
        a[k] = 1;
        src[k] = base_omegas[k];
    }
    NS_TRY(set_active(a));
    NS_TRY(gather(src.data()));
    NS_TRY(transform_W());
    NS_TRY(stream_function(stream_));   // P = Psi_b (kVel: U, V = its velocity)
    k_base_fields<T><<<dim3(kPtBlocks, S_), 256, 0, stream_>>>(f_, (T*)f_.Ub, (T*)f_.Vb, (T*)f_.DxOb, (T*)f_.DyOb);
    NS_LAUNCH_CHECK();
    NS_TRY(all_active());
    have_base_ = true;
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::step_linear(const double* v_in, double* v_out, int nsteps) {
    std::vector<const double*> pi(B_);
    std::vector<double*> po(B_);
    for (int m = 0; m < B_; ++m) {
        pi[m] = v_in + (size_t)m * n_;
        po[m] = v_out + (size_t)m * n_;
    }
    return step_linear_ptrs(pi.data(), po.data(), nsteps);
}

template <class T> int StepperImpl<T>::step_linear_ptrs(const double* const* in, double* const* out, int nsteps) {
    if (!have_base_) {
        set_error("linearised step requested before a base flow was set");
        return NSSTAB_ERR_INVALID_ARG;
    }
    std::vector<unsigned char> a(B_);
    for (int m = 0; m < B_; ++m) a[m] = in[m] != nullptr;
    NS_TRY(set_active(a));
    NS_TRY(gather(in));
    if (nsteps > 0) {
        NS_TRY(transform_W());
        NS_TRY(run_steps(nsteps, true, false, false));
    }
    return scatter(f_.W, out);
}

// dPhi_T(q)/dq v_in for the stepper's two members (one parameter set):
// member 0 marches q nonlinearly, member 1 marches v linearised about
// member 0's state of the same step (co-integration).  The base fields are
// overwritten along the way: a later linearised step needs a new base.
template <class T> int StepperImpl<T>::tangent(const double* q, const double* v_in, double* v_out, int nsteps) {
    if (B_ != 2 || S_ != 1) {
        set_error("tangent: needs a batch of two members and one parameter set");
        return NSSTAB_ERR_INVALID_ARG;
    }
    NS_TRY(alloc_base_fields());
    if (!tmask_) {
        NS_TRY(dalloc(&tmask_, 4));
        const unsigned char m4[4] = {1, 0, 0, 1};
        NS_CUDA(cudaMemcpy(tmask_, m4, 4, cudaMemcpyHostToDevice));
        clear_graphs();
    }
    have_base_ = false;
    NS_TRY(all_active());
    const double* src[2] = {q, v_in};
    NS_TRY(gather(src));
    if (nsteps > 0) {
        NS_TRY(transform_W());
        NS_TRY(run_steps(nsteps, false, false, false, true, true));
    }
    double* dst[2] = {nullptr, v_out};
    return scatter(f_.W, dst);
}

template <class T> int StepperImpl<T>::sumsq_diff(const T* a, const T* b, double* out) {
    k_diff_sumsq<T><<<dim3(kRedBlocks, B_), 256, 0, stream_>>>(a, b, n_, n_, red_);
    NS_LAUNCH_CHECK();
    NS_CUDA(cudaMemcpyAsync(red_host_, red_, (size_t)B_ * kRedBlocks * sizeof(double), cudaMemcpyDeviceToHost,
                            stream_));
    NS_CUDA(cudaStreamSynchronize(stream_));
    for (int m = 0; m < B_; ++m) {
        double s = 0.0;
        for (int b2 = 0; b2 < kRedBlocks; ++b2) s += red_host_[(size_t)m * kRedBlocks + b2];
        out[m] = s;
    }
    return NSSTAB_OK;
}

template <class T> int StepperImpl<T>::residual(const double* q, double* r) {
    if (!Wsave_) NS_TRY(dalloc(&Wsave_, (size_t)B_ * n_));
    NS_TRY(all_active());
    NS_TRY(gather_contig(q, B_));
    NS_CUDA(cudaMemcpyAsync(Wsave_, f_.W, (size_t)B_ * n_ * sizeof(T), cudaMemcpyDeviceToDevice, stream_));
    NS_TRY(transform_W());
    NS_TRY(run_steps(1, false, false, false));
    std::vector<double> ss(B_);
    NS_TRY(sumsq_diff(f_.W, Wsave_, ss.data()));
    const double dx = cfg_.Lx / nx_, dy = cfg_.Ly / ny_;
    for (int m = 0; m < B_; ++m) r[m] = std::sqrt(ss[m] * dx * dy) / cfg_.dt;
    return NSSTAB_OK;
}

template <class T>
int StepperImpl<T>::sfd(double* omega, double chi, double Delta, double tol, long max_steps, int check_every,
                        double* r_out, long* steps_out) {
    if (!f_.Y) {
        T* Y;
        NS_TRY(dalloc(&Y, (size_t)B_ * n_));
        f_.Y = Y;
    }
    if (!Wsave_) NS_TRY(dalloc(&Wsave_, (size_t)B_ * n_));
    if (!Nhsave_) NS_TRY(dalloc(&Nhsave_, (size_t)B_ * nc_));
    f_.sfd_k1 = (T)(cfg_.dt * chi);
    f_.sfd_k2 = (T)(cfg_.dt / Delta);
    clear_graphs();   // captured kernels carry the gains and the Y pointer by value
    NS_TRY(all_active());
    NS_TRY(gather_contig(omega, B_));
    NS_CUDA(cudaMemcpyAsync(f_.Y, f_.W, (size_t)B_ * n_ * sizeof(T), cudaMemcpyDeviceToDevice, stream_));
    NS_TRY(transform_W());
    const double dx = cfg_.Lx / nx_, dy = cfg_.Ly / ny_;
    long k = 0;
    std::vector<double> r(B_, INFINITY), ss(B_);
    int status = NSSTAB_NOT_CONVERGED;
    bool first_chunk = true;
    while (k < max_steps) {
        const long chunk = std::min<long>(check_every, max_steps - k);
        // the AB2 history continues across chunks: only the very first step is AB1
        NS_TRY(run_steps((int)chunk, false, true, true, first_chunk));
        first_chunk = false;
        k += chunk;
        // residual of the current X with one plain AB1 step, then restore the state
        NS_CUDA(cudaMemcpyAsync(Wsave_, f_.W, (size_t)B_ * n_ * sizeof(T), cudaMemcpyDeviceToDevice, stream_));
        NS_CUDA(cudaMemcpyAsync(Nhsave_, f_.Nh, (size_t)B_ * nc_ * sizeof(C), cudaMemcpyDeviceToDevice, stream_));
        NS_TRY(run_steps(1, false, false, false));
        NS_TRY(sumsq_diff(f_.W, Wsave_, ss.data()));
        bool all_ok = true, finite = true;
        for (int m = 0; m < B_; ++m) {
            r[m] = std::sqrt(ss[m] * dx * dy) / cfg_.dt;
            finite = finite && std::isfinite(r[m]);
            all_ok = all_ok && r[m] <= tol;
        }
        NS_CUDA(cudaMemcpyAsync(f_.W, Wsave_, (size_t)B_ * n_ * sizeof(T), cudaMemcpyDeviceToDevice, stream_));
        NS_CUDA(cudaMemcpyAsync(f_.Nh, Nhsave_, (size_t)B_ * nc_ * sizeof(C), cudaMemcpyDeviceToDevice, stream_));
        NS_TRY(transform_W());
        if (!finite) {
            status = NSSTAB_DIVERGED;
            break;
        }
        if (all_ok) {
            status = NSSTAB_OK;
            break;
        }
    }
    NS_TRY(scatter_contig(f_.W, omega));
    NS_CUDA(cudaStreamSynchronize(stream_));
    for (int m = 0; m < B_; ++m) r_out[m] = r[m];
    *steps_out = k;
    return status;
}

}  // namespace nsstab
