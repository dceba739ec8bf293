// Scalar-field operators of libjdft and the solvers built on them: full-box
// transforms of fields (I and J on ScalarField / ScalarFieldTilde, Sec. 2.1),
// the Hartree potential (periodic Coulomb kernel), LDA exchange-correlation,
// Pulay density mixing, the SCF driver around the band minimiser, and the
// linear dielectric (LinearPCM) Poisson solve of the paper's Listing 1.  The
// JDFTx paper names the Coulomb kernel (class Coulomb), the
// exchange-correlation functionals (class ExCorr) and self-consistency by
// Pulay mixing (class Pulay) in Sec. 2.1, SCF as the alternative to
// total-energy minimisation in Sec. 2.2, and gives the dielectric Poisson
// equation, the solvation energy and the CG solve of hessian(phi~) = rho~ in
// Sec. 2.1 (Eq. Poisson, Eq. Adiel, Listing 1); it prints no discretisation.
//
// Readings (shared with the test oracle only through the paper):
//   Fields    reciprocal-space fields are full complex boxes X(G), G = B iG
//             with frequencies folded to [-S/2, S/2) per axis;
//             I X (r_j) = sum_G X(G) exp(i G.r_j), J x = (1/N) sum_j x_j exp(-i G.r_j).
//   Hartree   nt = J n, V_H(G) = 4 pi nt(G) / |G|^2, V_H(0) = 0 (neutralising
//             background), V_H = I V_H(G); E_H = (Omega/2) sum_G 4 pi |nt(G)|^2 / |G|^2.
//   LDA       Slater exchange and the Perdew-Zunger 1981 fit of the
//             Ceperley-Alder correlation (Phys. Rev. B 23, 5048), unpolarised;
//             n <= 0 gives zero.  E_xc = (Omega/N) sum_j n_j e_xc(n_j).
//   Pulay     P. Pulay, Chem. Phys. Lett. 73, 393 (1980): coefficients that
//             minimise the norm of the combined residual under sum c = 1.
//   LinearPCM gradient = i G_d, divergence = sum_d i G_d, hessian(X) =
//             -(1/4 pi) div J(eps I(grad X)); preconditioned CG (preconditioner:
//             the Coulomb kernel) on G != 0 from phi~ = 0;
//             A_diel = (1/2) Re sum_G conj(phi~ - 4 pi rho~ / G^2) Omega rho~.
//
// Data layout: densities and potentials are real FP64 boxes, reciprocal-space
// fields complex FP64 boxes, j2 fastest.  The full-box transforms run one axis
// per launch: a block holds W lines of one axis in shared memory and
// transforms them with the Stockham passes of fft.cuh (FP64 throughout).  The
// Hartree chain is five launches: axis 2 (reading the real density), axis 1,
// axis 0 with the Coulomb kernel applied between its forward and inverse
// transforms (and the Hartree energy summed there), axis 1, and axis 2 whose
// epilogue writes the real potential (for the Kohn-Sham potential:
// V_ion + V_H + v_xc(n), with the exchange-correlation energy summed there).
// The dielectric hessian is five launches over three gradient boxes: axis 0
// forming i G_d X and transforming back, axis 1, axis 2 with the pointwise
// eps product between its inverse and forward transforms, axis 1, and axis 0
// summing i G_d (J ...)_d into the result (and the CG product d.Hd).
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "profile.cuh"

namespace jdft {
namespace {

constexpr int kFieldThreads = 256;
constexpr int kLineElems = 2048;   // complex elements per block and buffer
constexpr int kMaxHist = 16;        // Pulay pairs at most
constexpr int kReduceThreads = 256;
constexpr double kFourPi = 12.566370614359172953850573533118;

// Lines of one axis: line l = o * inner + i starts at o * ostride + i * istride,
// its elements es apart.
struct AxisGeom {
    int n;
    int W;                 // lines per block
    int64_t nlines;
    int64_t inner, ostride, istride, es;
};

struct FieldArgs {
    // Coulomb kernel pass: lattice and scale
    double B[9];           // column d = b_d, row-major
    int S[3];
    double invN;
    // Kohn-Sham epilogue
    const double* n;
    const double* vion;
    // per-block partial sums (E_H in the kernel pass, E_xc in the KS epilogue)
    double* partial;
    // complex stores are multiplied by `scale`; blockIdx.y selects one of a
    // batch of boxes `bstride` elements apart
    double scale;
    int64_t bstride;
};

AxisGeom axis_geom(const jdft_basis_s* b, int axis) {
    AxisGeom g;
    const int64_t S0 = b->S[0], S1 = b->S[1], S2 = b->S[2];
    g.n = b->S[axis];
    g.W = std::min(32, std::max(1, kLineElems / g.n));
    if (axis == 2) {
        g.nlines = S0 * S1; g.inner = g.nlines; g.istride = S2; g.ostride = 0; g.es = 1;
    } else if (axis == 1) {
        g.nlines = S0 * S2; g.inner = S2; g.istride = 1; g.ostride = S1 * S2; g.es = S2;
    } else {
        g.nlines = S1 * S2; g.inner = g.nlines; g.istride = 1; g.ostride = 0; g.es = S1 * S2;
    }
    return g;
}

__device__ __forceinline__ int fold(int m, int S) { return m < (S + 1) / 2 ? m : m - S; }

// Slater exchange + Perdew-Zunger correlation: energy per electron e and
// potential v at density n (both zero for n <= 0).
__device__ __forceinline__ void lda_pz(double n, double& e, double& v) {
    if (!(n > 0.0)) { e = 0.0; v = 0.0; return; }
    // one cube root and one reciprocal per point (FP64 transcendentals and
    // divisions are the cost of this epilogue on this GPU's FP64 rate)
    const double cx = -0.73855876638202240588423003065;   // -(3/4)(3/pi)^{1/3}
    const double kr = 0.62035049089940001666800681204778;  // (3/(4 pi))^{1/3}
    const double third = 1.0 / 3.0;
    const double c = cbrt(n);
    const double ex = cx * c;
    const double rs = kr / c;
    double ec, vc;
    if (rs >= 1.0) {
        const double g = -0.1423, b1 = 1.0529, b2 = 0.3334;
        const double sq = sqrt(rs);
        const double iden = 1.0 / (1.0 + b1 * sq + b2 * rs);
        ec = g * iden;
        // r_s de_c/dr_s = -g (b1 sqrt(r_s) / 2 + b2 r_s) / den^2
        const double rdec = -g * (0.5 * b1 * sq + b2 * rs) * iden * iden;
        vc = ec - third * rdec;
    } else {
        const double A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
        const double lr = log(rs);
        ec = A * lr + B + C * rs * lr + D * rs;
        // r_s de_c/dr_s = A + r_s (C (ln r_s + 1) + D)
        const double rdec = A + rs * (C * (lr + 1.0) + D);
        vc = ec - third * rdec;
    }
    e = ex + ec;
    v = (4.0 * third) * ex + vc;
}

// Sum over the block; thread 0 returns the total (others: partial values).
__device__ __forceinline__ double block_sum(double x) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;
}

// Shared-memory lines are stored with one padding element after every 32:
// element i of a buffer lives at pad_idx(i).  The radix-R passes write with
// stride R (and 8 Ns between groups), which without padding puts 4 to 16
// lanes of a warp on the same banks.
__host__ __device__ __forceinline__ int pad_idx(int i) { return i + (i >> 5); }
__host__ __device__ __forceinline__ int padded_len(int m) { return m + (m >> 5) + 1; }

// One Stockham pass of fft.cuh's transform over padded lines of length n.
template <typename T, int SIGN, int R>
__device__ __forceinline__ void stockham_pass_p(const c_t<T>* __restrict__ src, c_t<T>* __restrict__ dst, int nlines,
                                                int n, int Ns, const c_t<T>* __restrict__ tw) {
    const int nb = n / R;
    const int twstep = n / (Ns * R);
    const int total = nlines * nb;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int l = idx / nb;
        const int j = idx - l * nb;
        const int k = j % Ns;
        const int lb = l * n;
        c_t<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[pad_idx(lb + j + r * nb)];
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const c_t<T> w = tw[r * k * twstep];
                v[r] = (SIGN > 0) ? cmul(v[r], w) : cmulc(v[r], w);
            }
        }
        if (R == 2) dft2<T, SIGN>(v);
        if (R == 3) dft3<T, SIGN>(v);
        if (R == 4) dft4<T, SIGN>(v);
        if (R == 5) dft5<T, SIGN>(v);
        if (R == 8) dft8<T, SIGN>(v);
        const int ob = lb + (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[pad_idx(ob + r * Ns)] = v[r];
    }
}

// fft_lines (fft.cuh) on padded lines: nlines lines of length plan.n, line l
// at elements l * n.  Returns the buffer holding the result (block synchronised).
template <typename T, int SIGN>
__device__ c_t<T>* fft_lines_p(c_t<T>* a, c_t<T>* b, int nlines, const FftPlan& plan, const c_t<T>* __restrict__ tw) {
    int Ns = 1;
    const int n = plan.n;
    for (int p = 0; p < plan.npass; ++p) {
        const int R = plan.radix[p];
        switch (R) {
            case 2: stockham_pass_p<T, SIGN, 2>(a, b, nlines, n, Ns, tw); break;
            case 3: stockham_pass_p<T, SIGN, 3>(a, b, nlines, n, Ns, tw); break;
            case 4: stockham_pass_p<T, SIGN, 4>(a, b, nlines, n, Ns, tw); break;
            case 5: stockham_pass_p<T, SIGN, 5>(a, b, nlines, n, Ns, tw); break;
            default: stockham_pass_p<T, SIGN, 8>(a, b, nlines, n, Ns, tw); break;
        }
        __syncthreads();
        c_t<T>* t = a; a = b; b = t;
        Ns *= R;
    }
    return a;
}

enum { OUT_COMPLEX = 0, OUT_REAL = 1, OUT_KS = 2 };

// One axis of the full-box transform.  IN_REAL: the input is a real box
// (double), else complex.  KERNEL: apply the Coulomb kernel to the forward
// transform (SIGN = -1) and transform back along the same axis.  OUT: what
// the epilogue writes.
template <int SIGN, bool IN_REAL, bool KERNEL, int OUT>
__global__ void __launch_bounds__(kFieldThreads)
field_axis_kernel(const void* __restrict__ in, void* __restrict__ out, AxisGeom g, FftPlan plan,
                  const double2* __restrict__ tw, FieldArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int plen = padded_len(g.W * g.n);
    double2* bufA = reinterpret_cast<double2*>(smem_raw);
    double2* bufB = bufA + plen;
    int64_t* base = reinterpret_cast<int64_t*>(bufB + plen);
    if (!IN_REAL && OUT == OUT_COMPLEX && blockIdx.y > 0) {
        in = reinterpret_cast<const double2*>(in) + blockIdx.y * a.bstride;
        out = reinterpret_cast<double2*>(out) + blockIdx.y * a.bstride;
    }
    const int64_t l0 = (int64_t)blockIdx.x * g.W;
    const int64_t left = g.nlines - l0;
    const int nw = left < g.W ? (int)left : g.W;
    const int n = g.n;
    if (threadIdx.x < nw) {
        const int64_t l = l0 + threadIdx.x;
        const int64_t o = l / g.inner;
        base[threadIdx.x] = o * g.ostride + (l - o * g.inner) * g.istride;
    }
    __syncthreads();
    const int total = nw * n;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int w, t;
        if (g.es == 1) { w = idx / n; t = idx - w * n; } else { t = idx / nw; w = idx - t * nw; }
        const int64_t addr = base[w] + (int64_t)t * g.es;
        double2 v;
        if (IN_REAL) { v.x = reinterpret_cast<const double*>(in)[addr]; v.y = 0.0; }
        else v = reinterpret_cast<const double2*>(in)[addr];
        bufA[pad_idx(w * n + t)] = v;
    }
    __syncthreads();
    double2* res = fft_lines_p<double, SIGN>(bufA, bufB, nw, plan, tw);
    double part = 0.0;
    if (KERNEL) {
        // lines of axis 0: l = j1 * S2 + j2, position t = frequency index along
        // axis 0; each line's axis-1 and axis-2 part of G formed once (over the
        // W * 3 doubles after `base`)
        double* lineG = reinterpret_cast<double*>(base + g.W);
        if (threadIdx.x < nw) {
            const int64_t l = l0 + threadIdx.x;
            const int m1 = (int)(l / a.S[2]), m2 = (int)(l - (int64_t)m1 * a.S[2]);
            const double f1 = fold(m1, a.S[1]), f2 = fold(m2, a.S[2]);
            for (int c = 0; c < 3; ++c) lineG[3 * threadIdx.x + c] = f1 * a.B[3 * c + 1] + f2 * a.B[3 * c + 2];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int w = idx / n, t = idx - w * n;
            const double f0 = fold(t, a.S[0]);
            const double gx = f0 * a.B[0] + lineG[3 * w];
            const double gy = f0 * a.B[3] + lineG[3 * w + 1];
            const double gz = f0 * a.B[6] + lineG[3 * w + 2];
            const double G2 = gx * gx + gy * gy + gz * gz;
            const double K = G2 > 0.0 ? kFourPi / G2 : 0.0;
            double2 x = res[pad_idx(idx)];
            x.x *= a.invN; x.y *= a.invN;
            part += K * (x.x * x.x + x.y * x.y);
            res[pad_idx(idx)] = make_double2(K * x.x, K * x.y);
        }
        __syncthreads();
        double2* other = (res == bufA) ? bufB : bufA;
        res = fft_lines_p<double, -SIGN>(res, other, nw, plan, tw);
    }
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int w, t;
        if (g.es == 1) { w = idx / n; t = idx - w * n; } else { t = idx / nw; w = idx - t * nw; }
        const int64_t addr = base[w] + (int64_t)t * g.es;
        const double2 v = res[pad_idx(w * n + t)];
        if (OUT == OUT_COMPLEX) {
            reinterpret_cast<double2*>(out)[addr] = make_double2(a.scale * v.x, a.scale * v.y);
        } else if (OUT == OUT_REAL) {
            reinterpret_cast<double*>(out)[addr] = v.x;
        } else {
            const double nj = a.n[addr];
            double e, vx;
            lda_pz(nj, e, vx);
            reinterpret_cast<double*>(out)[addr] = a.vion[addr] + v.x + vx;
            part += nj * e;
        }
    }
    if (KERNEL || OUT == OUT_KS) {
        const double s = block_sum(part);
        if (threadIdx.x == 0) a.partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kFieldThreads)
lda_kernel(const double* __restrict__ n, double* __restrict__ vxc, double* __restrict__ partial, int64_t N) {
    double part = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        double e, v;
        lda_pz(n[j], e, v);
        if (vxc) vxc[j] = v;
        part += n[j] * e;
    }
    const double s = block_sum(part);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[k] (+)= scale * sum_b partial[b * stride + k] in a fixed order
// (deterministic); one block per k.
__global__ void __launch_bounds__(kReduceThreads)
reduce_partials_kernel(const double* __restrict__ partial, int count, int stride, double scale,
                       double* __restrict__ out, int accumulate) {
    const int k = blockIdx.x;
    double t = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) t += partial[(int64_t)i * stride + k];
    const double s = block_sum(t);
    if (threadIdx.x == 0) out[k] = (accumulate ? out[k] : 0.0) + scale * s;
}

// SCF bookkeeping over the box: partial sums of n_out (vks - vion) and of
// (n_out - n_in)^2, two per block.
__global__ void __launch_bounds__(kFieldThreads)
scf_sums_kernel(const double* __restrict__ nout, const double* __restrict__ nin, const double* __restrict__ vks,
                const double* __restrict__ vion, double* __restrict__ partial, int64_t N) {
    double dc = 0.0, rr = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const double no = nout[j];
        dc += no * (vks[j] - vion[j]);
        const double r = no - nin[j];
        rr += r * r;
    }
    const double s0 = block_sum(dc);
    const double s1 = block_sum(rr);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s0;
        partial[2 * blockIdx.x + 1] = s1;
    }
}

int reduce_grid(int64_t N) {
    int64_t g = (N + kFieldThreads * 4 - 1) / (kFieldThreads * 4);
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

// Field workspace of the basis: `nbox` complex boxes, then the partial sums.
struct FieldWork {
    double2* box;
    double* partial;     // kPartialMax doubles
};
constexpr int64_t kPartialMax = 1 << 17;

jdft_status field_work(jdft_basis_s* b, FieldWork* w, int nbox = 1) {
    jdft_status s = ensure_ws(b->fieldwork, (size_t)nbox * b->N * sizeof(double2) + kPartialMax * sizeof(double));
    if (s) return s;
    w->box = reinterpret_cast<double2*>(b->fieldwork.ptr);
    w->partial = reinterpret_cast<double*>(w->box + (size_t)nbox * b->N);
    return JDFT_OK;
}

size_t axis_smem(const AxisGeom& g) {
    // two padded buffers, the line bases and (for the Coulomb-kernel pass) 3 doubles a line
    return (size_t)2 * padded_len(g.W * g.n) * sizeof(double2) + (size_t)g.W * sizeof(int64_t) +
           (size_t)3 * g.W * sizeof(double);
}

template <int SIGN, bool IN_REAL, bool KERNEL, int OUT>
jdft_status launch_axis(const char* name, jdft_basis_s* b, int axis, const void* in, void* out, const FieldArgs& a,
                        cudaStream_t st, int* nblocks = nullptr, int batch = 1) {
    const AxisGeom g = axis_geom(b, axis);
    const int64_t grid = (g.nlines + g.W - 1) / g.W;
    if ((KERNEL || OUT == OUT_KS) && grid > kPartialMax)
        return set_error(JDFT_ERR_ARG, "box too large for the field workspace's partial sums");
    const size_t smem = axis_smem(g);
    auto kern = field_axis_kernel<SIGN, IN_REAL, KERNEL, OUT>;
    JDFT_CUDA_TRY(set_smem_attr((const void*)kern, smem));
    const FftPlan plan = b->plan[axis];
    {
        Trace tr_(name, st);
        kern<<<dim3((unsigned)grid, (unsigned)batch), kFieldThreads, smem, st>>>(in, out, g, plan,
                                                                                b->tw64 + plan.tw_offset, a);
    }
    if (nblocks) *nblocks = (int)grid;
    return check_launch(name);
}

FieldArgs field_args(const jdft_basis_s* b, double* partial) {
    FieldArgs a;
    for (int i = 0; i < 9; ++i) a.B[i] = b->B[i];
    for (int d = 0; d < 3; ++d) a.S[d] = b->S[d];
    a.invN = 1.0 / (double)b->N;
    a.n = nullptr;
    a.vion = nullptr;
    a.partial = partial;
    a.scale = 1.0;
    a.bstride = b->N;
    return a;
}

jdft_status launch_reduce(const double* partial, int count, int stride, int nout, double scale, double* out,
                          bool accumulate, cudaStream_t st) {
    {
        Trace tr_("reduce_partials", st);
        reduce_partials_kernel<<<nout, kReduceThreads, 0, st>>>(partial, count, stride, scale, out, accumulate ? 1 : 0);
    }
    return check_launch("reduce_partials");
}

// V = V_H[n] (OUT_REAL) or V_ion + V_H[n] + v_xc[n] (OUT_KS); energies[0] = E_H,
// energies[1] = E_xc (KS only) when energies is not NULL.
template <int OUT>
jdft_status hartree_chain(jdft_basis_s* b, const double* n, const double* vion, double* V, double* energies,
                          cudaStream_t st) {
    FieldWork w;
    jdft_status s = field_work(b, &w);
    if (s) return s;
    // the two partial-sum regions: E_H (kernel pass) and E_xc (last pass)
    const int64_t half = kPartialMax / 2;
    FieldArgs a = field_args(b, w.partial);
    int nb_h = 0, nb_x = 0;
    for (int axis = 0; axis < 3; axis += 2) {
        const AxisGeom g = axis_geom(b, axis);
        if ((g.nlines + g.W - 1) / g.W > half) return set_error(JDFT_ERR_ARG, "box too large for the partial sums");
    }
    if ((s = launch_axis<-1, true, false, OUT_COMPLEX>("field_fft_axis2", b, 2, n, w.box, a, st))) return s;
    if ((s = launch_axis<-1, false, false, OUT_COMPLEX>("field_fft_axis1", b, 1, w.box, w.box, a, st))) return s;
    if ((s = launch_axis<-1, false, true, OUT_COMPLEX>("hartree_kernel_axis0", b, 0, w.box, w.box, a, st, &nb_h)))
        return s;
    if ((s = launch_axis<+1, false, false, OUT_COMPLEX>("field_fft_axis1", b, 1, w.box, w.box, a, st))) return s;
    FieldArgs e = a;
    e.n = n;
    e.vion = vion;
    e.partial = w.partial + half;
    if (OUT == OUT_KS) {
        if ((s = launch_axis<+1, false, false, OUT_KS>("ks_potential_axis2", b, 2, w.box, V, e, st, &nb_x))) return s;
    } else {
        if ((s = launch_axis<+1, false, false, OUT_REAL>("field_fft_axis2", b, 2, w.box, V, e, st))) return s;
    }
    if (energies) {
        if ((s = launch_reduce(w.partial, nb_h, 1, 1, 0.5 * b->omega, energies, false, st))) return s;
        if (OUT == OUT_KS)
            if ((s = launch_reduce(w.partial + half, nb_x, 1, 1, b->omega / (double)b->N, energies + 1, false, st)))
                return s;
    }
    return JDFT_OK;
}

// ---------------------------------------------------------------------------
// Pulay mixing
// ---------------------------------------------------------------------------

// Store the new pair in ring slot s (n_in, R = n_out - n_in) and sum, per
// block, R . R_i for the stored slots i < count (slot s included).  Block row
// y of the grid takes slots [kPulayGroup y, kPulayGroup (y + 1)) (few
// accumulators a thread, so many blocks fit an SM); row 0 also stores the pair.
constexpr int kPulayGroup = 4;

__global__ void __launch_bounds__(kFieldThreads)
pulay_store_kernel(const double* __restrict__ nin, const double* __restrict__ nout, double* __restrict__ Nbuf,
                   double* __restrict__ Rbuf, int slot, int count, int64_t N, double* __restrict__ partial) {
    const int i0 = blockIdx.y * kPulayGroup;
    const bool store = blockIdx.y == 0;
    double acc[kPulayGroup];
#pragma unroll
    for (int q = 0; q < kPulayGroup; ++q) acc[q] = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const double x = nin[j];
        const double r = nout[j] - x;
        if (store) {
            Nbuf[(int64_t)slot * N + j] = x;
            Rbuf[(int64_t)slot * N + j] = r;
        }
#pragma unroll
        for (int q = 0; q < kPulayGroup; ++q) {
            const int i = i0 + q;
            if (i < count) acc[q] += r * (i == slot ? r : Rbuf[(int64_t)i * N + j]);
        }
    }
#pragma unroll
    for (int q = 0; q < kPulayGroup; ++q) {
        if (i0 + q < count) {
            const double s = block_sum(acc[q]);
            if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kMaxHist + i0 + q] = s;
        }
    }
}

// Sum the partial dots into row and column `slot` of A (hist x hist), then
// solve the bordered system over the stored pairs, oldest first, dropping the
// oldest pair while a pivot falls below 1e-13 max |A_ii|.  coef[slot] for the
// pairs used, 0 for the rest; meta[0] = pairs used.
__global__ void __launch_bounds__(kMaxHist)
pulay_solve_kernel(const double* __restrict__ partial, int nblk, double* __restrict__ A, int hist, int slot,
                   int count, double* __restrict__ coef, int* __restrict__ meta) {
    const int i = threadIdx.x;
    if (i < count) {
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += partial[(int64_t)b * kMaxHist + i];
        A[slot * hist + i] = t;
        A[i * hist + slot] = t;
    }
    __syncthreads();
    if (i != 0) return;
    int order[kMaxHist];
    for (int a = 0; a < count; ++a) order[a] = ((slot - (count - 1) + a) % hist + hist) % hist;
    for (int k = 0; k < hist; ++k) coef[k] = 0.0;
    double M[kMaxHist + 1][kMaxHist + 2];
    double x[kMaxHist + 1];
    for (int first = 0; first < count; ++first) {
        const int m = count - first;
        double dmax = 0.0;
        for (int r = 0; r < m; ++r) dmax = fmax(dmax, fabs(A[order[first + r] * hist + order[first + r]]));
        const double thresh = 1e-13 * dmax;
        for (int r = 0; r <= m; ++r)
            for (int c = 0; c <= m + 1; ++c) M[r][c] = 0.0;
        for (int r = 0; r < m; ++r) {
            for (int c = 0; c < m; ++c) M[r][c] = A[order[first + r] * hist + order[first + c]];
            M[r][m] = 1.0;
            M[m][r] = 1.0;
        }
        M[m][m + 1] = 1.0;
        bool ok = true;
        for (int col = 0; col <= m && ok; ++col) {
            int p = col;
            for (int r = col + 1; r <= m; ++r)
                if (fabs(M[r][col]) > fabs(M[p][col])) p = r;
            if (fabs(M[p][col]) <= thresh) { ok = false; break; }
            if (p != col)
                for (int c = 0; c <= m + 1; ++c) { const double t = M[p][c]; M[p][c] = M[col][c]; M[col][c] = t; }
            for (int r = col + 1; r <= m; ++r) {
                const double f = M[r][col] / M[col][col];
                for (int c = col; c <= m + 1; ++c) M[r][c] -= f * M[col][c];
            }
        }
        if (!ok && m > 1) continue;
        if (!ok) {
            coef[order[first]] = 1.0;
        } else {
            for (int r = m; r >= 0; --r) {
                double t = M[r][m + 1];
                for (int c = r + 1; c <= m; ++c) t -= M[r][c] * x[c];
                x[r] = t / M[r][r];
            }
            for (int r = 0; r < m; ++r) coef[order[first + r]] = x[r];
        }
        meta[0] = m;
        return;
    }
}

__global__ void __launch_bounds__(kFieldThreads)
pulay_mix_kernel(const double* __restrict__ Nbuf, const double* __restrict__ Rbuf, const double* __restrict__ coef,
                 int count, double alpha, int64_t N, double* __restrict__ out) {
    // the coefficients in shared memory (read uniformly), not in registers
    __shared__ double c[kMaxHist];
    if (threadIdx.x < kMaxHist) c[threadIdx.x] = threadIdx.x < count ? coef[threadIdx.x] : 0.0;
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int i = 0; i < count; ++i) {
            const double ci = c[i];
            if (ci != 0.0) t += ci * (Nbuf[(int64_t)i * N + j] + alpha * Rbuf[(int64_t)i * N + j]);
        }
        out[j] = t;
    }
}


// ---------------------------------------------------------------------------
// LinearPCM: hessian(X) = -(1/4 pi) div J(eps I(grad X)) on reciprocal-space boxes
// ---------------------------------------------------------------------------

struct GArgs {
    double B[9];   // column d = b_d, row-major
    int S[3];
};

// Cartesian component c of G for folded frequency indices (m0, m1, m2).
__device__ __forceinline__ double g_comp(const GArgs& q, int c, double f0, double f1, double f2) {
    return f0 * q.B[3 * c] + f1 * q.B[3 * c + 1] + f2 * q.B[3 * c + 2];
}

// |G|^2 of box slot j in precision T (boxes hold fewer than 2^31 points).
template <typename T>
__device__ __forceinline__ T g2_of_index(const GArgs& q, int64_t jj) {
    const int j = (int)jj;
    const int plane = q.S[1] * q.S[2];
    const int m0 = j / plane;
    const int rem = j - m0 * plane;
    const int m1 = rem / q.S[2], m2 = rem - m1 * q.S[2];
    const T f0 = (T)fold(m0, q.S[0]), f1 = (T)fold(m1, q.S[1]), f2 = (T)fold(m2, q.S[2]);
    T g2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T gc = f0 * (T)q.B[3 * c] + f1 * (T)q.B[3 * c + 1] + f2 * (T)q.B[3 * c + 2];
        g2 += gc * gc;
    }
    return g2;
}

// Coulomb kernel 4 pi / |G|^2 of slot j in precision T (0 at G = 0).
template <typename T>
__device__ __forceinline__ T coulomb_of_index(const GArgs& q, int64_t j) {
    const T g2 = g2_of_index<T>(q, j);
    return g2 > (T)0 ? (T)kFourPi / g2 : (T)0;
}

__device__ __forceinline__ void line_index(const AxisGeom& g, int nw, int idx, int& w, int& t) {
    if (g.es == 1) { w = idx / g.n; t = idx - w * g.n; } else { t = idx / nw; w = idx - t * nw; }
}

// Complex element of type T from double parts, and back.
template <typename T> __device__ __forceinline__ c_t<T> cx(double re, double im) { return mk<T>((T)re, (T)im); }

// One axis pass over complex boxes of type T (batch of boxes via blockIdx.y,
// bstride apart), in place or out of place.
template <typename T, int SIGN>
__global__ void __launch_bounds__(kFieldThreads)
field_axis_c_kernel(const c_t<T>* __restrict__ in, c_t<T>* __restrict__ out, AxisGeom g, FftPlan plan,
                    const c_t<T>* __restrict__ tw, int64_t bstride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int plen = padded_len(g.W * g.n);
    c_t<T>* bufA = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* bufB = bufA + plen;
    int64_t* base = reinterpret_cast<int64_t*>(bufB + plen);
    in += blockIdx.y * bstride;
    out += blockIdx.y * bstride;
    const int64_t l0 = (int64_t)blockIdx.x * g.W;
    const int64_t left = g.nlines - l0;
    const int nw = left < g.W ? (int)left : g.W;
    const int n = g.n;
    if (threadIdx.x < nw) {
        const int64_t l = l0 + threadIdx.x;
        const int64_t o = l / g.inner;
        base[threadIdx.x] = o * g.ostride + (l - o * g.inner) * g.istride;
    }
    __syncthreads();
    const int total = nw * n;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int w, t;
        line_index(g, nw, idx, w, t);
        bufA[pad_idx(w * n + t)] = in[base[w] + (int64_t)t * g.es];
    }
    __syncthreads();
    const c_t<T>* res = fft_lines_p<T, SIGN>(bufA, bufB, nw, plan, tw);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int w, t;
        line_index(g, nw, idx, w, t);
        out[base[w] + (int64_t)t * g.es] = res[pad_idx(w * n + t)];
    }
}

// Axis 0 of the gradient's inverse transform: for each line of X (reciprocal
// space; lines along axis 0, l = m1 S2 + m2), Y_c = I_0 (i G_c X), c = 0, 1, 2
// (boxes bstride apart).
template <typename T>
__global__ void __launch_bounds__(kFieldThreads)
pcm_grad_axis0_kernel(const c_t<T>* __restrict__ X, c_t<T>* __restrict__ Y, AxisGeom g, FftPlan plan,
                      const c_t<T>* __restrict__ tw, GArgs q, int64_t bstride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int plen = padded_len(g.W * g.n);
    c_t<T>* bufX = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* bufA = bufX + plen;
    c_t<T>* bufB = bufA + plen;
    int64_t* base = reinterpret_cast<int64_t*>(bufB + plen);
    const int64_t l0 = (int64_t)blockIdx.x * g.W;
    const int64_t left = g.nlines - l0;
    const int nw = left < g.W ? (int)left : g.W;
    const int n = g.n;
    T* lineG = reinterpret_cast<T*>(base + g.W);                  // per line: sum over axes 1, 2 of G_c
    if (threadIdx.x < nw) {
        const int64_t l = l0 + threadIdx.x;
        base[threadIdx.x] = l;                                      // axis 0: line l starts at l
        const int m1 = (int)(l / q.S[2]), m2 = (int)(l - (int64_t)m1 * q.S[2]);
        const double f1 = fold(m1, q.S[1]), f2 = fold(m2, q.S[2]);
        for (int c = 0; c < 3; ++c) lineG[3 * threadIdx.x + c] = (T)(f1 * q.B[3 * c + 1] + f2 * q.B[3 * c + 2]);
    }
    __syncthreads();
    const int total = nw * n;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int w, t;
        line_index(g, nw, idx, w, t);
        bufX[pad_idx(w * n + t)] = X[base[w] + (int64_t)t * g.es];
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
        const T b0 = (T)q.B[3 * c];
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int w = idx / n, t = idx - w * n;
            const T G = (T)fold(t, q.S[0]) * b0 + lineG[3 * w + c];
            const c_t<T> x = bufX[pad_idx(idx)];
            bufA[pad_idx(idx)] = mk<T>(-G * x.y, G * x.x);
        }
        __syncthreads();
        const c_t<T>* res = fft_lines_p<T, +1>(bufA, bufB, nw, plan, tw);
        c_t<T>* Yc = Y + c * bstride;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int w, t;
            line_index(g, nw, idx, w, t);
            Yc[base[w] + (int64_t)t * g.es] = res[pad_idx(w * n + t)];
        }
        __syncthreads();
    }
}

// Axis 2 (contiguous lines) of each gradient box (blockIdx.y): inverse
// transform, pointwise product with eps(r), forward transform, in place.
template <typename T>
__global__ void __launch_bounds__(kFieldThreads)
pcm_eps_axis2_kernel(c_t<T>* __restrict__ Y, const T* __restrict__ eps, AxisGeom g, FftPlan plan,
                     const c_t<T>* __restrict__ tw, int64_t bstride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c_t<T>* bufA = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* bufB = bufA + padded_len(g.W * g.n);
    Y += blockIdx.y * bstride;
    const int64_t l0 = (int64_t)blockIdx.x * g.W;
    const int64_t left = g.nlines - l0;
    const int nw = left < g.W ? (int)left : g.W;
    const int n = g.n;
    const int total = nw * n;
    const int64_t off = l0 * n;   // axis 2: line l starts at l * S2, contiguous
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) bufA[pad_idx(idx)] = Y[off + idx];
    __syncthreads();
    c_t<T>* res = fft_lines_p<T, +1>(bufA, bufB, nw, plan, tw);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const T e = eps[off + idx];
        res[pad_idx(idx)].x *= e;
        res[pad_idx(idx)].y *= e;
    }
    __syncthreads();
    c_t<T>* other = (res == bufA) ? bufB : bufA;
    res = fft_lines_p<T, -1>(res, other, nw, plan, tw);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) Y[off + idx] = res[pad_idx(idx)];
}

// Axis 0 of the forward transforms and the divergence: out = scale *
// sum_c i G_c F_0(Y_c); with din, per-block partial sums of Re conj(din) out.
template <typename T>
__global__ void __launch_bounds__(kFieldThreads)
pcm_div_axis0_kernel(const c_t<T>* __restrict__ Y, const c_t<T>* __restrict__ din, c_t<T>* __restrict__ out,
                     AxisGeom g, FftPlan plan, const c_t<T>* __restrict__ tw, GArgs q, int64_t bstride,
                     double scale, double* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int plen = padded_len(g.W * g.n);
    c_t<T>* acc = reinterpret_cast<c_t<T>*>(smem_raw);
    c_t<T>* bufA = acc + plen;
    c_t<T>* bufB = bufA + plen;
    int64_t* base = reinterpret_cast<int64_t*>(bufB + plen);
    const int64_t l0 = (int64_t)blockIdx.x * g.W;
    const int64_t left = g.nlines - l0;
    const int nw = left < g.W ? (int)left : g.W;
    const int n = g.n;
    T* lineG = reinterpret_cast<T*>(base + g.W);                  // per line: sum over axes 1, 2 of G_c
    if (threadIdx.x < nw) {
        const int64_t l = l0 + threadIdx.x;
        base[threadIdx.x] = l;
        const int m1 = (int)(l / q.S[2]), m2 = (int)(l - (int64_t)m1 * q.S[2]);
        const double f1 = fold(m1, q.S[1]), f2 = fold(m2, q.S[2]);
        for (int c = 0; c < 3; ++c) lineG[3 * threadIdx.x + c] = (T)(f1 * q.B[3 * c + 1] + f2 * q.B[3 * c + 2]);
    }
    const int total = nw * n;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) acc[pad_idx(idx)] = mk<T>(0, 0);
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
        const c_t<T>* Yc = Y + c * bstride;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int w, t;
            line_index(g, nw, idx, w, t);
            bufA[pad_idx(w * n + t)] = Yc[base[w] + (int64_t)t * g.es];
        }
        __syncthreads();
        const c_t<T>* res = fft_lines_p<T, -1>(bufA, bufB, nw, plan, tw);
        const T b0 = (T)q.B[3 * c];
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int w = idx / n, t = idx - w * n;
            const T G = (T)fold(t, q.S[0]) * b0 + lineG[3 * w + c];
            const c_t<T> y = res[pad_idx(idx)];
            acc[pad_idx(idx)].x -= G * y.y;
            acc[pad_idx(idx)].y += G * y.x;
        }
        __syncthreads();
    }
    T part = 0;
    const T sc = (T)scale;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int w, t;
        line_index(g, nw, idx, w, t);
        const int64_t addr = base[w] + (int64_t)t * g.es;
        const c_t<T> a = acc[pad_idx(w * n + t)];
        const c_t<T> v = mk<T>(sc * a.x, sc * a.y);
        out[addr] = v;
        if (din) {
            const c_t<T> dv = din[addr];
            part += dv.x * v.x + dv.y * v.y;
        }
    }
    if (din) {
        const double t = block_sum((double)part);
        if (threadIdx.x == 0) partial[blockIdx.x] = t;
    }
}

// CG start: r = rho~ without its G = 0 term (converted to T), x = 0 (if x),
// d = K r; partial sums of |r|^2 and r.Kr (two per block).
template <typename T>
__global__ void __launch_bounds__(kFieldThreads)
pcm_init_kernel(const double2* __restrict__ rho, c_t<T>* __restrict__ x, c_t<T>* __restrict__ r,
                c_t<T>* __restrict__ d, GArgs q, int64_t N, double* __restrict__ partial) {
    double rr = 0.0, rz = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const double G2 = g2_of_index<double>(q, j);
        const double K = G2 > 0.0 ? kFourPi / G2 : 0.0;
        const double2 v = G2 > 0.0 ? rho[j] : make_double2(0.0, 0.0);
        const c_t<T> vt = cx<T>(v.x, v.y);
        r[j] = vt;
        if (x) x[j] = mk<T>(0, 0);
        d[j] = mk<T>((T)K * vt.x, (T)K * vt.y);
        const double a = (double)vt.x * vt.x + (double)vt.y * vt.y;
        rr += a;
        rz += K * a;
    }
    const double s0 = block_sum(rr);
    const double s1 = block_sum(rz);
    if (threadIdx.x == 0) { partial[2 * blockIdx.x] = s0; partial[2 * blockIdx.x + 1] = s1; }
}

// x += alpha d, r -= alpha Hd with alpha = rz / dHd (device scalars); partial
// sums of |r|^2 and r.Kr of the new residual.
template <typename T>
__global__ void __launch_bounds__(kFieldThreads)
pcm_update_kernel(c_t<T>* __restrict__ x, c_t<T>* __restrict__ r, const c_t<T>* __restrict__ d,
                  const c_t<T>* __restrict__ Hd, const double* __restrict__ rz, const double* __restrict__ dHd,
                  GArgs q, int64_t N, double* __restrict__ partial) {
    const T alpha = (T)(*rz / *dHd);
    T rr = 0, rzn = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const c_t<T> dv = d[j], hv = Hd[j];
        c_t<T> xv = x[j], rv = r[j];
        xv.x += alpha * dv.x; xv.y += alpha * dv.y;
        rv.x -= alpha * hv.x; rv.y -= alpha * hv.y;
        x[j] = xv;
        r[j] = rv;
        const T K = coulomb_of_index<T>(q, j);
        const T a = rv.x * rv.x + rv.y * rv.y;
        rr += a;
        rzn += K * a;
    }
    const double s0 = block_sum((double)rr);
    const double s1 = block_sum((double)rzn);
    if (threadIdx.x == 0) { partial[2 * blockIdx.x] = s0; partial[2 * blockIdx.x + 1] = s1; }
}

// d = K r + beta d, beta = rz_new / rz_old (device scalars).
template <typename T>
__global__ void __launch_bounds__(kFieldThreads)
pcm_direction_kernel(const c_t<T>* __restrict__ r, c_t<T>* __restrict__ d, const double* __restrict__ rz_new,
                     const double* __restrict__ rz_old, GArgs q, int64_t N) {
    const T beta = (T)(*rz_new / *rz_old);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const T K = coulomb_of_index<T>(q, j);
        const c_t<T> rv = r[j], dv = d[j];
        d[j] = mk<T>(K * rv.x + beta * dv.x, K * rv.y + beta * dv.y);
    }
}

// Mixed solve, refinement step: x += e (FP32 correction), then (after the
// FP64 hessian of x into Hx) r = rho~ - Hx on G != 0 with partial |r|^2.
__global__ void __launch_bounds__(kFieldThreads)
pcm_accumulate_kernel(double2* __restrict__ x, const float2* __restrict__ e, int64_t N) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const float2 ev = e[j];
        double2 xv = x[j];
        xv.x += (double)ev.x;
        xv.y += (double)ev.y;
        x[j] = xv;
    }
}

__global__ void __launch_bounds__(kFieldThreads)
pcm_residual_kernel(const double2* __restrict__ rho, const double2* __restrict__ Hx, double2* __restrict__ r, GArgs q,
                    int64_t N, double* __restrict__ partial) {
    double rr = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const double G2 = g2_of_index<double>(q, j);
        double2 v = make_double2(0.0, 0.0);
        if (G2 > 0.0) {
            const double2 a = rho[j], h = Hx[j];
            v = make_double2(a.x - h.x, a.y - h.y);
        }
        r[j] = v;
        rr += v.x * v.x + v.y * v.y;
    }
    const double s = block_sum(rr);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Residual replacement: r32 = r64 (the FP64 residual) in the block type, with
// partial sums of |r|^2 and r.Kr (two per block).
template <typename T>
__global__ void __launch_bounds__(kFieldThreads)
pcm_refresh_kernel(const double2* __restrict__ r64, c_t<T>* __restrict__ r, GArgs q, int64_t N,
                   double* __restrict__ partial) {
    double rr = 0.0, rz = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = r64[j];
        const c_t<T> vt = cx<T>(v.x, v.y);
        r[j] = vt;
        const double a = (double)vt.x * vt.x + (double)vt.y * vt.y;
        rr += a;
        rz += (double)coulomb_of_index<T>(q, j) * a;
    }
    const double s0 = block_sum(rr);
    const double s1 = block_sum(rz);
    if (threadIdx.x == 0) { partial[2 * blockIdx.x] = s0; partial[2 * blockIdx.x + 1] = s1; }
}

__global__ void __launch_bounds__(kFieldThreads)
to_float_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t N) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x)
        b[j] = (float)a[j];
}

// Partial sums of Re conj(phi~ - K rho~) rho~ over G != 0.
__global__ void __launch_bounds__(kFieldThreads)
pcm_energy_kernel(const double2* __restrict__ phi, const double2* __restrict__ rho, GArgs q, int64_t N,
                  double* __restrict__ partial) {
    double e = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const double G2 = g2_of_index<double>(q, j);
        if (G2 > 0.0) {
            const double K = kFourPi / G2;
            const double2 p = phi[j], v = rho[j];
            e += (p.x - K * v.x) * v.x + (p.y - K * v.y) * v.y;
        }
    }
    const double s = block_sum(e);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

GArgs g_args(const jdft_basis_s* b) {
    GArgs q;
    for (int i = 0; i < 9; ++i) q.B[i] = b->B[i];
    for (int d = 0; d < 3; ++d) q.S[d] = b->S[d];
    return q;
}

template <typename T> const c_t<T>* twiddles_of(const jdft_basis_s* b);
template <> const double2* twiddles_of<double>(const jdft_basis_s* b) { return b->tw64; }
template <> const float2* twiddles_of<float>(const jdft_basis_s* b) { return b->tw32; }

// hessian of X into out (out must overlap neither X nor the three gradient
// boxes Yg); with din, partial sums of Re conj(din) out into partial.
template <typename T>
jdft_status pcm_hessian(jdft_basis_s* b, const T* eps, const c_t<T>* X, c_t<T>* out, c_t<T>* Yg,
                        const c_t<T>* din, double* partial, int* nblocks, cudaStream_t st) {
    const GArgs q = g_args(b);
    const AxisGeom g0 = axis_geom(b, 0), g1 = axis_geom(b, 1), g2 = axis_geom(b, 2);
    const int64_t grid0 = (g0.nlines + g0.W - 1) / g0.W;
    const int64_t grid1 = (g1.nlines + g1.W - 1) / g1.W;
    const int64_t grid2 = (g2.nlines + g2.W - 1) / g2.W;
    if (grid0 > kPartialMax - 16) return set_error(JDFT_ERR_ARG, "box too large for the partial sums");
    const size_t e = sizeof(c_t<T>);
    const size_t smem3 = (size_t)3 * padded_len(g0.W * g0.n) * e + g0.W * sizeof(int64_t) +
                         (size_t)3 * g0.W * sizeof(T);
    const size_t smem1 = (size_t)2 * padded_len(g1.W * g1.n) * e + g1.W * sizeof(int64_t);
    const size_t smem2 = (size_t)2 * padded_len(g2.W * g2.n) * e;
    JDFT_CUDA_TRY(set_smem_attr((const void*)pcm_grad_axis0_kernel<T>, smem3));
    JDFT_CUDA_TRY(set_smem_attr((const void*)pcm_div_axis0_kernel<T>, smem3));
    JDFT_CUDA_TRY(set_smem_attr((const void*)pcm_eps_axis2_kernel<T>, smem2));
    JDFT_CUDA_TRY(set_smem_attr((const void*)field_axis_c_kernel<T, +1>, smem1));
    JDFT_CUDA_TRY(set_smem_attr((const void*)field_axis_c_kernel<T, -1>, smem1));
    const FftPlan p0 = b->plan[0], p1 = b->plan[1], p2 = b->plan[2];
    const c_t<T>* tw = twiddles_of<T>(b);
    const int64_t N = b->N;
    {
        Trace tr_("pcm_grad_axis0", st);
        pcm_grad_axis0_kernel<T><<<(unsigned)grid0, kFieldThreads, smem3, st>>>(X, Yg, g0, p0, tw + p0.tw_offset, q,
                                                                                 N);
    }
    jdft_status s = check_launch("pcm_grad_axis0");
    if (s) return s;
    {
        Trace tr_("field_fft_axis1_batch", st);
        field_axis_c_kernel<T, +1><<<dim3((unsigned)grid1, 3), kFieldThreads, smem1, st>>>(Yg, Yg, g1, p1,
                                                                                          tw + p1.tw_offset, N);
    }
    if ((s = check_launch("field_fft_axis1_batch"))) return s;
    {
        Trace tr_("pcm_eps_axis2", st);
        pcm_eps_axis2_kernel<T><<<dim3((unsigned)grid2, 3), kFieldThreads, smem2, st>>>(Yg, eps, g2, p2,
                                                                                       tw + p2.tw_offset, N);
    }
    if ((s = check_launch("pcm_eps_axis2"))) return s;
    {
        Trace tr_("field_fft_axis1_batch", st);
        field_axis_c_kernel<T, -1><<<dim3((unsigned)grid1, 3), kFieldThreads, smem1, st>>>(Yg, Yg, g1, p1,
                                                                                          tw + p1.tw_offset, N);
    }
    if ((s = check_launch("field_fft_axis1_batch"))) return s;
    {
        Trace tr_("pcm_div_axis0", st);
        pcm_div_axis0_kernel<T><<<(unsigned)grid0, kFieldThreads, smem3, st>>>(
            Yg, din, out, g0, p0, tw + p0.tw_offset, q, N, -1.0 / (kFourPi * (double)N), partial);
    }
    if (nblocks) *nblocks = (int)grid0;
    return check_launch("pcm_div_axis0");
}

// Preconditioned CG on hessian(x) = r0 for boxes of type T, from x = 0:
// r0 is read from rho (FP64; its G = 0 term dropped).  Stops when
// |r| <= rel_tol |r0| or after max_iter hessians.  Vectors: x, r, d, Hd, Yg
// (3 boxes).  sc: 8 device doubles of scratch.  Returns the iterations taken
// and |r| / |r0| at exit.
template <typename T>
jdft_status pcm_cg(jdft_basis_s* b, const T* eps, const double2* rho, c_t<T>* x, c_t<T>* r, c_t<T>* d,
                   c_t<T>* Hd, c_t<T>* Yg, double* partial, double* sc, double rel_tol, int max_iter,
                   int* iters, double* rel_res, double* r0norm, cudaStream_t st) {
    const int64_t N = b->N;
    const int grid = reduce_grid(N);
    const GArgs q = g_args(b);
    jdft_status s;
    {
        Trace tr_("pcm_init", st);
        pcm_init_kernel<T><<<grid, kFieldThreads, 0, st>>>(rho, x, r, d, q, N, partial);
    }
    if ((s = check_launch("pcm_init"))) return s;
    if ((s = launch_reduce(partial, grid, 2, 2, 1.0, sc + 2, false, st))) return s;
    double host[2];
    JDFT_CUDA_TRY(cudaMemcpyAsync(host, sc + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    JDFT_CUDA_TRY(cudaStreamSynchronize(st));
    const double bnorm = std::sqrt(host[0]);
    if (r0norm) *r0norm = bnorm;
    double res = 0.0;
    int it = 0;
    if (bnorm > 0.0) {
        res = 1.0;
        for (it = 0; it < max_iter;) {
            int nb0 = 0;
            if ((s = pcm_hessian<T>(b, eps, d, Hd, Yg, d, partial, &nb0, st))) return s;
            if ((s = launch_reduce(partial, nb0, 1, 1, 1.0, sc, false, st))) return s;
            double* old = sc + 2 + 2 * (it & 1);
            double* nw = sc + 2 + 2 * ((it + 1) & 1);
            {
                Trace tr_("pcm_update", st);
                pcm_update_kernel<T><<<grid, kFieldThreads, 0, st>>>(x, r, d, Hd, old + 1, sc, q, N, partial);
            }
            if ((s = check_launch("pcm_update"))) return s;
            if ((s = launch_reduce(partial, grid, 2, 2, 1.0, nw, false, st))) return s;
            JDFT_CUDA_TRY(cudaMemcpyAsync(host, nw, sizeof(double), cudaMemcpyDeviceToHost, st));
            JDFT_CUDA_TRY(cudaStreamSynchronize(st));
            ++it;
            res = std::sqrt(host[0]) / bnorm;
            if (!(res > rel_tol)) break;
            {
                Trace tr_("pcm_direction", st);
                pcm_direction_kernel<T><<<grid, kFieldThreads, 0, st>>>(r, d, nw + 1, old + 1, q, N);
            }
            if ((s = check_launch("pcm_direction"))) return s;
        }
    }
    *iters = it;
    *rel_res = res;
    return JDFT_OK;
}

}  // namespace
}  // namespace jdft

struct jdft_pulay_s {
    int64_t n = 0;
    int hist = 0;
    double alpha = 0.5;
    int count = 0;      // stored pairs
    int head = -1;      // slot of the newest pair
    int nblk = 0;
    int device = 0;
    double* Nbuf = nullptr;
    double* Rbuf = nullptr;
    double* A = nullptr;
    double* partial = nullptr;
    double* coef = nullptr;
    int* meta = nullptr;
};

using namespace jdft;

extern "C" {

jdft_status jdft_hartree(jdft_basis_t b, const double* n, double* vh, double* energy, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && n && vh, "null argument");
    JDFT_CHECK_ARG(n != vh, "n and vh must not overlap");
    return hartree_chain<OUT_REAL>(b, n, nullptr, vh, energy, (cudaStream_t)stream);
}

jdft_status jdft_xc_lda(jdft_basis_t b, const double* n, double* vxc, double* energy, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && n, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    FieldWork w;
    jdft_status s = field_work(b, &w);
    if (s) return s;
    const int grid = reduce_grid(b->N);
    {
        Trace tr_("lda_xc", st);
        lda_kernel<<<grid, kFieldThreads, 0, st>>>(n, vxc, w.partial, b->N);
    }
    if ((s = check_launch("lda_xc"))) return s;
    if (energy) return launch_reduce(w.partial, grid, 1, 1, b->omega / (double)b->N, energy, false, st);
    return JDFT_OK;
}

jdft_status jdft_ks_potential(jdft_basis_t b, const double* n, const double* vion, double* vks, double* energies,
                              void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && n && vion && vks, "null argument");
    JDFT_CHECK_ARG(n != vks && vion != vks, "vks must not overlap n or vion");
    return hartree_chain<OUT_KS>(b, n, vion, vks, energies, (cudaStream_t)stream);
}

jdft_status jdft_pulay_create(int64_t n, int history, double alpha, jdft_pulay_t* out) {
    clear_error();
    JDFT_CHECK_ARG(out, "null output handle");
    *out = nullptr;
    JDFT_CHECK_ARG(n >= 1, "n must be >= 1");
    JDFT_CHECK_ARG(history >= 1 && history <= kMaxHist, "history must be in [1, 16]");
    JDFT_CHECK_ARG(alpha > 0 && alpha <= 1 && std::isfinite(alpha), "alpha must be in (0, 1]");
    jdft_pulay_s* p = new jdft_pulay_s();
    p->n = n;
    p->hist = history;
    p->alpha = alpha;
    p->nblk = reduce_grid(n);
    cudaGetDevice(&p->device);
    cudaError_t e = cudaSuccess;
    size_t vec = (size_t)history * n * sizeof(double);
    if (e == cudaSuccess) e = cudaMalloc(&p->Nbuf, vec);
    if (e == cudaSuccess) e = cudaMalloc(&p->Rbuf, vec);
    if (e == cudaSuccess) e = cudaMalloc(&p->A, (size_t)history * history * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->partial, (size_t)p->nblk * kMaxHist * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->coef, (size_t)kMaxHist * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->meta, sizeof(int));
    if (e != cudaSuccess) {
        jdft_pulay_destroy(p);
        return set_error(e == cudaErrorMemoryAllocation ? JDFT_ERR_OOM : JDFT_ERR_CUDA,
                         std::string("jdft_pulay_create: ") + cudaGetErrorString(e));
    }
    *out = p;
    return JDFT_OK;
}

jdft_status jdft_pulay_destroy(jdft_pulay_t p) {
    if (!p) return JDFT_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaFree(p->Nbuf); cudaFree(p->Rbuf); cudaFree(p->A); cudaFree(p->partial); cudaFree(p->coef);
    cudaFree(p->meta);
    cudaSetDevice(prev);
    delete p;
    return JDFT_OK;
}

jdft_status jdft_pulay_reset(jdft_pulay_t p) {
    clear_error();
    JDFT_CHECK_ARG(p, "null handle");
    p->count = 0;
    p->head = -1;
    return JDFT_OK;
}

jdft_status jdft_pulay_step(jdft_pulay_t p, const double* n_in, const double* n_out, double* n_next, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(p && n_in && n_out && n_next, "null argument");
    JDFT_CHECK_ARG(n_next != n_out, "n_next must not be n_out");
    cudaStream_t st = (cudaStream_t)stream;
    const int slot = (p->head + 1) % p->hist;
    const int count = std::min(p->count + 1, p->hist);
    {
        Trace tr_("pulay_store", st);
        const dim3 grid(p->nblk, (count + kPulayGroup - 1) / kPulayGroup);
        pulay_store_kernel<<<grid, kFieldThreads, 0, st>>>(n_in, n_out, p->Nbuf, p->Rbuf, slot, count, p->n,
                                                           p->partial);
    }
    jdft_status s = check_launch("pulay_store");
    if (s) return s;
    {
        Trace tr_("pulay_solve", st);
        pulay_solve_kernel<<<1, kMaxHist, 0, st>>>(p->partial, p->nblk, p->A, p->hist, slot, count, p->coef, p->meta);
    }
    if ((s = check_launch("pulay_solve"))) return s;
    {
        Trace tr_("pulay_mix", st);
        pulay_mix_kernel<<<p->nblk, kFieldThreads, 0, st>>>(p->Nbuf, p->Rbuf, p->coef, count, p->alpha, p->n,
                                                            n_next);
    }
    if ((s = check_launch("pulay_mix"))) return s;
    p->head = slot;
    p->count = count;
    return JDFT_OK;
}

jdft_status jdft_pulay_used(jdft_pulay_t p, int* used, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(p && used, "null argument");
    *used = 0;
    if (p->count == 0) return JDFT_OK;
    JDFT_CUDA_TRY(cudaMemcpyAsync(used, p->meta, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    JDFT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return JDFT_OK;
}

jdft_status jdft_scf(jdft_basis_t b, void* const* C, int ldc, int nb, const double* vion, double* n_r, double* eigs,
                     const jdft_scf_opts* opts, jdft_scf_report* report, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && C && vion && n_r && opts && report, "null argument");
    JDFT_CHECK_ARG(nb >= 1, "nb must be >= 1");
    for (int ik = 0; ik < b->nk; ++ik) {
        JDFT_CHECK_ARG(C[ik], "null coefficient block");
        JDFT_CHECK_ARG(nb <= b->ks[ik].npw && ldc >= b->ks[ik].npw, "bad block shape");
    }
    JDFT_CHECK_ARG(opts->history >= 0 && opts->history <= kMaxHist, "history must be in [0, 16]");
    JDFT_CHECK_ARG(opts->alpha >= 0 && opts->alpha <= 1, "alpha must be in [0, 1]");
    JDFT_CHECK_ARG(opts->max_iter >= 0 && opts->band_max_iter >= 0, "negative iteration limit");
    JDFT_CHECK_ARG(opts->precond != JDFT_PRECOND_MLP || opts->mlp, "MLP preconditioner needs weights");
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    *report = jdft_scf_report();
    const double tolE = opts->tol_energy > 0 ? opts->tol_energy : 1e-8;
    const double tolN = opts->tol_density > 0 ? opts->tol_density : 1e-6;
    const int maxit = opts->max_iter > 0 ? opts->max_iter : 100;
    const int hist = opts->history > 0 ? opts->history : 8;
    const double alpha = opts->alpha > 0 ? opts->alpha : 0.5;
    const double f = opts->occupation > 0 ? opts->occupation : 2.0;
    const int64_t N = b->N;
    jdft_min_opts mo;
    mo.tol = opts->band_tol > 0 ? opts->band_tol : 1e-9;
    mo.max_iter = opts->band_max_iter > 0 ? opts->band_max_iter : 1000;
    mo.precond = opts->precond;
    mo.prec = opts->prec;
    mo.switch_tol = 0.0;
    mo.occupation = f;
    mo.mlp = opts->mlp;

    // working fields: n_in, n_out, vks, scratch potential, occupations, scalars
    double* wk = nullptr;
    const size_t nd = (size_t)4 * N + nb + 8;
    JDFT_CUDA_TRY(cudaMalloc(&wk, nd * sizeof(double)));
    double *nin = wk, *nout = wk + N, *vks = wk + 2 * N, *vtmp = wk + 3 * N, *focc = wk + 4 * N;
    double* sc = focc + nb;            // [E_H, E_xc, dc, rr]
    double* eig_d = nullptr;
    jdft_pulay_t mix = nullptr;
    std::vector<double> fh(nb, f), eh((size_t)b->nk * nb), scal(4);
    jdft_status s = JDFT_OK;
    double E = 0.0, Eprev = 0.0, res = 0.0;
    auto fail = [&](jdft_status st_) {
        cudaStreamSynchronize(st);
        cudaFree(wk);
        cudaFree(eig_d);
        jdft_pulay_destroy(mix);
        return st_;
    };
    if (cudaMalloc(&eig_d, (size_t)b->nk * nb * sizeof(double)) != cudaSuccess)
        return fail(set_error(JDFT_ERR_OOM, "jdft_scf: eigenvalue buffer"));
    if ((s = jdft_pulay_create(N, hist, alpha, &mix))) return fail(s);
    if (cudaMemcpyAsync(focc, fh.data(), nb * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(nin, 0, N * sizeof(double), st) != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_scf: set-up copies"));
    // starting density: the orthonormalised starting blocks
    for (int ik = 0; ik < b->nk; ++ik) {
        if ((s = jdft_orthonormalize(b, ik, C[ik], ldc, nb, JDFT_FP64, stream))) return fail(s);
        if ((s = jdft_density(b, ik, C[ik], ldc, focc, nb, nin, JDFT_FP64, stream))) return fail(s);
    }
    const int grid = reduce_grid(N);
    FieldWork w;
    if ((s = field_work(b, &w))) return fail(s);
    bool converged = false;
    int it = 0;
    const double band_tol = mo.tol;
    const double factor = opts->band_tol_factor == 0.0 ? 0.01 : opts->band_tol_factor;
    for (it = 1; it <= maxit; ++it) {
        // loose band solves while the density is far from self-consistency
        mo.tol = factor < 0.0 ? band_tol : std::max(band_tol, it == 1 ? 1e-3 : std::min(1e-3, factor * res));
        if ((s = jdft_ks_potential(b, nin, vion, vks, nullptr, stream))) return fail(s);
        if ((s = jdft_set_potential(b, vks, stream))) return fail(s);
        double Eband = 0.0;
        for (int ik = 0; ik < b->nk; ++ik) {
            jdft_min_report mr;
            s = jdft_minimize_bands(b, ik, C[ik], ldc, nb, &mo, eig_d + (size_t)ik * nb, &mr, stream);
            report->band_iterations += mr.iterations;
            // an inner solve that hit its limit still gives usable orbitals: the
            // outer loop goes on (its own test decides convergence)
            if (s == JDFT_ERR_NOT_CONVERGED) { report->band_unconverged += 1; s = JDFT_OK; }
            if (s) return fail(s);
        }
        if (cudaMemcpyAsync(eh.data(), eig_d, eh.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return fail(set_error(JDFT_ERR_CUDA, "jdft_scf: eigenvalue copy"));
        if (cudaMemsetAsync(nout, 0, N * sizeof(double), st) != cudaSuccess)
            return fail(set_error(JDFT_ERR_CUDA, "jdft_scf: memset"));
        for (int ik = 0; ik < b->nk; ++ik)
            if ((s = jdft_density(b, ik, C[ik], ldc, focc, nb, nout, JDFT_FP64, stream))) return fail(s);
        {
            Trace tr_("scf_sums", st);
            scf_sums_kernel<<<grid, kFieldThreads, 0, st>>>(nout, nin, vks, vion, w.partial, N);
        }
        if ((s = check_launch("scf_sums"))) return fail(s);
        if ((s = launch_reduce(w.partial, grid, 2, 2, 1.0, sc + 2, false, st))) return fail(s);
        // E_H and E_xc of the output density (its potential is not needed)
        if ((s = jdft_ks_potential(b, nout, vion, vtmp, sc, stream))) return fail(s);
        if (cudaMemcpyAsync(scal.data(), sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(set_error(JDFT_ERR_CUDA, "jdft_scf: scalar copy"));
        for (int ik = 0; ik < b->nk; ++ik)
            for (int i = 0; i < nb; ++i) Eband += b->kweight[ik] * f * eh[(size_t)ik * nb + i];
        const double dOmega = b->omega / (double)N;
        const double Edc = -dOmega * scal[2];
        E = Eband + Edc + scal[0] + scal[1];
        res = std::sqrt(dOmega * scal[3]);
        report->band_energy = Eband;
        report->double_counting = Edc;
        report->hartree = scal[0];
        report->xc = scal[1];
        report->energy = E;
        report->residual = res;
        report->iterations = it;
        if (it > 1 && std::fabs(E - Eprev) < tolE && res < tolN) { converged = true; break; }
        Eprev = E;
        if (it == maxit) break;
        if ((s = jdft_pulay_step(mix, nin, nout, nin, stream))) return fail(s);
    }
    // outputs: the last output density and eigenvalues; the basis keeps V_KS of the last input density
    if (cudaMemcpyAsync(n_r, nout, N * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_scf: density copy"));
    if (eigs && cudaMemcpyAsync(eigs, eig_d, eh.size() * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_scf: eigenvalue copy"));
    report->converged = converged ? 1 : 0;
    fail(JDFT_OK);
    report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!converged) return set_error(JDFT_ERR_NOT_CONVERGED, "SCF reached its iteration limit");
    return JDFT_OK;
}

jdft_status jdft_field_I(jdft_basis_t b, const void* X, void* x, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && X && x, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    FieldArgs a = field_args(b, nullptr);
    jdft_status s;
    if ((s = launch_axis<+1, false, false, OUT_COMPLEX>("field_fft_axis0", b, 0, X, x, a, st))) return s;
    if ((s = launch_axis<+1, false, false, OUT_COMPLEX>("field_fft_axis1", b, 1, x, x, a, st))) return s;
    return launch_axis<+1, false, false, OUT_COMPLEX>("field_fft_axis2", b, 2, x, x, a, st);
}

jdft_status jdft_field_J(jdft_basis_t b, const void* x, void* X, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && X && x, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    FieldArgs a = field_args(b, nullptr);
    jdft_status s;
    if ((s = launch_axis<-1, false, false, OUT_COMPLEX>("field_fft_axis2", b, 2, x, X, a, st))) return s;
    if ((s = launch_axis<-1, false, false, OUT_COMPLEX>("field_fft_axis1", b, 1, X, X, a, st))) return s;
    a.scale = 1.0 / (double)b->N;
    return launch_axis<-1, false, false, OUT_COMPLEX>("field_fft_axis0", b, 0, X, X, a, st);
}

jdft_status jdft_pcm_hessian(jdft_basis_t b, const double* eps, const void* phi_t, void* out_t, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && eps && phi_t && out_t, "null argument");
    JDFT_CHECK_ARG(phi_t != out_t, "out_t must not overlap phi_t");
    FieldWork w;
    jdft_status s = field_work(b, &w, 3);
    if (s) return s;
    return pcm_hessian<double>(b, eps, (const double2*)phi_t, (double2*)out_t, w.box, nullptr, w.partial, nullptr,
                               (cudaStream_t)stream);
}

jdft_status jdft_pcm_solve(jdft_basis_t b, const double* eps, const void* rho_t, void* phi_t, double tol,
                           int max_iter, jdft_prec prec, jdft_pcm_report* report, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b && eps && rho_t && phi_t && report, "null argument");
    JDFT_CHECK_ARG(rho_t != phi_t, "phi_t must not overlap rho_t");
    JDFT_CHECK_ARG(tol > 0 && max_iter >= 1, "bad tolerance or iteration limit");
    JDFT_CHECK_ARG(prec == JDFT_FP64 || prec == JDFT_FP32, "prec must be JDFT_FP64 or JDFT_FP32");
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    *report = jdft_pcm_report();
    const int64_t N = b->N;
    double2* x = (double2*)phi_t;
    const double2* rho = (const double2*)rho_t;
    const GArgs q = g_args(b);
    const int grid = reduce_grid(N);
    FieldWork w;
    jdft_status s;
    double res = 0.0;
    int its = 0, its64 = 0;
    if (prec == JDFT_FP64) {
        // boxes: three gradient components, r, d, Hd
        if ((s = field_work(b, &w, 6))) return s;
        double* sc = w.partial + kPartialMax - 8;
        if ((s = pcm_cg<double>(b, eps, rho, x, w.box + 3 * N, w.box + 4 * N, w.box + 5 * N, w.box, w.partial, sc, tol,
                                max_iter, &its, &res, nullptr, st)))
            return s;
        its64 = its;
    } else {
        // FP32 corrections, FP64 residuals: FP64 boxes Yg (3), r, Hx; FP32 boxes
        // Yg (3), r, d, Hd, e (8 bytes each, 4 per FP64 box slot pair) and eps.
        const int64_t f64 = 5, f32_boxes = 7;
        const int64_t nbox = f64 + (f32_boxes + 1) / 2 + 1;     // FP32 boxes packed two per slot, eps in one
        if ((s = field_work(b, &w, (int)nbox))) return s;
        double2 *Yg64 = w.box, *r64 = w.box + 3 * N, *Hx = w.box + 4 * N;
        float2* f = reinterpret_cast<float2*>(w.box + f64 * N);
        float2 *Yg32 = f, *r32 = f + 3 * N, *d32 = f + 4 * N, *Hd32 = f + 5 * N, *e32 = f + 6 * N;
        float* eps32 = reinterpret_cast<float*>(f + 8 * N);
        double* sc = w.partial + kPartialMax - 8;
        {
            Trace tr_("to_float", st);
            to_float_kernel<<<grid, kFieldThreads, 0, st>>>(eps, eps32, N);
        }
        if ((s = check_launch("to_float"))) return s;
        // x = 0, r = rho~ (G != 0): the residual of x = 0
        {
            Trace tr_("pcm_residual", st);
            JDFT_CUDA_TRY(cudaMemsetAsync(x, 0, N * sizeof(double2), st));
            JDFT_CUDA_TRY(cudaMemsetAsync(Hx, 0, N * sizeof(double2), st));
            pcm_residual_kernel<<<grid, kFieldThreads, 0, st>>>(rho, Hx, r64, q, N, w.partial);
        }
        if ((s = check_launch("pcm_residual"))) return s;
        if ((s = launch_reduce(w.partial, grid, 1, 1, 1.0, sc + 7, false, st))) return s;
        double host = 0.0;
        JDFT_CUDA_TRY(cudaMemcpyAsync(&host, sc + 7, sizeof(double), cudaMemcpyDeviceToHost, st));
        JDFT_CUDA_TRY(cudaStreamSynchronize(st));
        const double bnorm = std::sqrt(host);
        res = bnorm > 0.0 ? 1.0 : 0.0;
        // One CG on the correction equation in FP32 (e32, r32, d32), its residual
        // replaced by the FP64 one whenever it has fallen by kReplace since the
        // last replacement or below half the tolerance: x += e, r = rho~ - H x in
        // FP64, the direction kept (reliable updates).
        const double kReplace = 1e-4;
        if (res > tol) {
            {
                Trace tr_("pcm_init", st);
                pcm_init_kernel<float><<<grid, kFieldThreads, 0, st>>>(r64, e32, r32, d32, q, N, w.partial);
            }
            if ((s = check_launch("pcm_init"))) return s;
            if ((s = launch_reduce(w.partial, grid, 2, 2, 1.0, sc + 2, false, st))) return s;
            JDFT_CUDA_TRY(cudaMemcpyAsync(&host, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
            JDFT_CUDA_TRY(cudaStreamSynchronize(st));
        }
        double rref = std::sqrt(host);
        int k = 0;                 // parity of the (|r|^2, r.Kr) slots
        while (res > tol && its < max_iter) {
            int nb0 = 0;
            if ((s = pcm_hessian<float>(b, eps32, d32, Hd32, Yg32, d32, w.partial, &nb0, st))) return s;
            if ((s = launch_reduce(w.partial, nb0, 1, 1, 1.0, sc, false, st))) return s;
            double* old = sc + 2 + 2 * (k & 1);
            double* nw = sc + 2 + 2 * ((k + 1) & 1);
            {
                Trace tr_("pcm_update", st);
                pcm_update_kernel<float><<<grid, kFieldThreads, 0, st>>>(e32, r32, d32, Hd32, old + 1, sc, q, N,
                                                                         w.partial);
            }
            if ((s = check_launch("pcm_update"))) return s;
            if ((s = launch_reduce(w.partial, grid, 2, 2, 1.0, nw, false, st))) return s;
            JDFT_CUDA_TRY(cudaMemcpyAsync(&host, nw, sizeof(double), cudaMemcpyDeviceToHost, st));
            JDFT_CUDA_TRY(cudaStreamSynchronize(st));
            ++its;
            ++k;
            // update when the residual has fallen by kReplace, or is near the
            // tolerance itself (so the solve stops close to it)
            if (std::sqrt(host) <= std::max(kReplace * rref, 0.5 * tol * bnorm) || its >= max_iter) {
                {
                    Trace tr_("pcm_accumulate", st);
                    pcm_accumulate_kernel<<<grid, kFieldThreads, 0, st>>>(x, e32, N);
                }
                if ((s = check_launch("pcm_accumulate"))) return s;
                JDFT_CUDA_TRY(cudaMemsetAsync(e32, 0, N * sizeof(float2), st));
                if ((s = pcm_hessian<double>(b, eps, x, Hx, Yg64, nullptr, w.partial, nullptr, st))) return s;
                ++its64;
                {
                    Trace tr_("pcm_residual", st);
                    pcm_residual_kernel<<<grid, kFieldThreads, 0, st>>>(rho, Hx, r64, q, N, w.partial);
                }
                if ((s = check_launch("pcm_residual"))) return s;
                if ((s = launch_reduce(w.partial, grid, 1, 1, 1.0, sc + 7, false, st))) return s;
                JDFT_CUDA_TRY(cudaMemcpyAsync(&host, sc + 7, sizeof(double), cudaMemcpyDeviceToHost, st));
                JDFT_CUDA_TRY(cudaStreamSynchronize(st));
                const double prev = res;
                res = std::sqrt(host) / bnorm;
                if (!(res > tol) || !(res < prev)) break;   // converged, or the FP32 corrections are exhausted
                {
                    Trace tr_("pcm_refresh", st);
                    pcm_refresh_kernel<float><<<grid, kFieldThreads, 0, st>>>(r64, r32, q, N, w.partial);
                }
                if ((s = check_launch("pcm_refresh"))) return s;
                if ((s = launch_reduce(w.partial, grid, 2, 2, 1.0, nw, false, st))) return s;
                JDFT_CUDA_TRY(cudaMemcpyAsync(&host, nw, sizeof(double), cudaMemcpyDeviceToHost, st));
                JDFT_CUDA_TRY(cudaStreamSynchronize(st));
                rref = std::sqrt(host);
            }
            {
                Trace tr_("pcm_direction", st);
                pcm_direction_kernel<float><<<grid, kFieldThreads, 0, st>>>(r32, d32, nw + 1, old + 1, q, N);
            }
            if ((s = check_launch("pcm_direction"))) return s;
        }
    }
    {
        Trace tr_("pcm_energy", st);
        pcm_energy_kernel<<<grid, kFieldThreads, 0, st>>>(x, rho, q, N, w.partial);
    }
    if ((s = check_launch("pcm_energy"))) return s;
    double* sc = w.partial + kPartialMax - 8;
    if ((s = launch_reduce(w.partial, grid, 1, 1, 0.5 * b->omega, sc + 6, false, st))) return s;
    double A = 0.0;
    JDFT_CUDA_TRY(cudaMemcpyAsync(&A, sc + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
    JDFT_CUDA_TRY(cudaStreamSynchronize(st));
    report->iterations = its;
    report->fp64_hessians = its64;
    report->residual = res;
    report->converged = (res <= tol) ? 1 : 0;
    report->A_diel = A;
    report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!report->converged) return set_error(JDFT_ERR_NOT_CONVERGED, "dielectric CG reached its iteration limit");
    return JDFT_OK;
}

}  // extern "C"
