// k_matvec_tp.cu -- the TMA-fed operator-product kernels (Sec. 4.1): a
// producer warp streams each element row's blocks as column units into a
// shared-memory ring with bulk copies, and consumer threads (one or two rows
// of the element row each) accumulate the s stage sums from shared memory.
// Variant forms 5-10 of the launch table in k_matvec.cu.
#include <algorithm>
#include <type_traits>

#include "matvec.cuh"
#include "tma.cuh"

namespace irk_mv {
namespace {

// ---------------------------------------------------------------------------
// TMA-fed variant with the block size at compile time (double-float).  A CTA
// holds G row groups of B consumer threads (whole warps) and one producer
// warp; lane g of the producer warp streams group g's work as units of CK
// block columns, one bulk copy each (CK B entries, contiguous in the
// column-major layout), into a ring of NU units per group, and with the
// first unit of every block one more copy of the s B stage values of the
// block's neighbour into a ring of NX stage-value slots; each unit completes
// on its "full" mbarrier.  The consumers read only shared memory (the HBM
// stream and the neighbours' stage values arrive ahead of them without
// holding registers) and release a unit on its "empty" mbarrier (B
// arrivals).  Refilling a unit's slot waits for the unit NU places earlier,
// which lies past the last unit of the block NX places earlier, so a
// stage-value slot is refilled only after its block is done (NX below).
// Rows: group g of CTA b takes rows (b + t gridDim.x) G + g, t = 0, 1, ...
// Every accumulator sees the columns in ascending order and folds after the
// same columns as every other variant: the result is theirs, bit for bit.
// Waits are bounded; on a timeout the kernel records IRK_DEV_ERR_TIMEOUT,
// the producer stops issuing and waits for its copies in flight, and every
// thread leaves.
template <int S, int B, int CK, int NU, int R = 1, int GO = 0, int PW = 1>
struct TpShape {
    static_assert(R == 1 || (R == 2 && B % 2 == 0), "two rows per thread need an even block size");
    static constexpr int BT = B / R;                     // consumer threads per group
    // row groups per CTA: whole warps of groups within 256 threads, or (GO >
    // 0) as many groups as fit in about GO consumer threads
    static constexpr int G = GO > 0 ? (GO / BT > 0 ? GO / BT : 1) : sp_groups(BT);
    static constexpr int CONS = (G * BT + 31) / 32 * 32;  // consumer threads (whole warps)
    static constexpr int GPW = (G + PW - 1) / PW;         // groups per producer warp
    static constexpr int THREADS = CONS + 32 * PW;       // and the producer warps
    static constexpr int UPB = (B + CK - 1) / CK;        // units per block
    static constexpr int NX = 1 + (NU - 1 + UPB - 1) / UPB;  // stage-value slots per group
    static constexpr int UNIT = CK * B * 8;              // a multiple of 16 for even B
    static constexpr int XSLOT = S * B * 8;
    static constexpr int HEADER = ((2 * NU * G * 8 + 16 + 127) / 128) * 128;
    static constexpr int GROUP = NU * UNIT + NX * XSLOT;  // a multiple of 16
    static constexpr int SMEM = HEADER + G * GROUP;
};

// acc[l] += sum over NC columns (from c0) of B_entry * x_l (thread row a),
// two columns at a time; the fold points (every eighth column, the block's
// last) are the second column of a pair (B even)
template <int S, int B, bool XF, int NC>
__device__ __forceinline__ void tp_consume(df_acc (&acc)[S], const unsigned char *unit, const float *X, int c0,
                                           int a) {
    const float2 *Jc = reinterpret_cast<const float2 *>(unit);
#pragma unroll
    for (int c = 0; c < NC; c += 2) {
        const float2 b0 = Jc[c * B + a], b1 = Jc[(c + 1) * B + a];
#pragma unroll
        for (int l = 0; l < S; ++l) {
            const float4 xv = *reinterpret_cast<const float4 *>(X + 2 * (l * B + c0 + c));
            if (XF) {
                df_acc_fma_f(acc[l], df_make(b0.x, b0.y), xv.x);
                df_acc_fma_f(acc[l], df_make(b1.x, b1.y), xv.z);
            } else {
                df_acc_fma(acc[l], df_make(b0.x, b0.y), df_make(xv.x, xv.y));
                df_acc_fma(acc[l], df_make(b1.x, b1.y), df_make(xv.z, xv.w));
            }
        }
        if (fold_after(c0 + c + 1, B))
#pragma unroll
            for (int l = 0; l < S; ++l) df_acc_renorm(acc[l]);
    }
}

// tp_consume for two rows per thread (a, a + 1: one 16-byte load per column),
// each accumulator pair in the two lanes of packed binary32 instructions
template <int S, int B, bool XF, int NC>
__device__ __forceinline__ void tp_consume2(df_acc2 (&acc)[S], const unsigned char *unit, const float *X, int c0,
                                            int a) {
    const float4 *Jc = reinterpret_cast<const float4 *>(unit);
#pragma unroll
    for (int c = 0; c < NC; c += 2) {
        const float4 b0 = Jc[(c * B + a) >> 1], b1 = Jc[((c + 1) * B + a) >> 1];
        const f32x2 h0 = f2_pack(b0.x, b0.z), l0 = f2_pack(b0.y, b0.w);
        const f32x2 h1 = f2_pack(b1.x, b1.z), l1 = f2_pack(b1.y, b1.w);
        const f32x2 n0 = f2_neg(h0), n1 = f2_neg(h1);  // once per column for all stages
#pragma unroll
        for (int l = 0; l < S; ++l) {
            const float4 xv = *reinterpret_cast<const float4 *>(X + 2 * (l * B + c0 + c));
            if (XF) {
                df_acc2_fma_f(acc[l], h0, n0, l0, f2_pack(xv.x, xv.x));
                df_acc2_fma_f(acc[l], h1, n1, l1, f2_pack(xv.z, xv.z));
            } else {
                df_acc2_fma(acc[l], h0, n0, l0, f2_pack(xv.x, xv.x), f2_pack(xv.y, xv.y));
                df_acc2_fma(acc[l], h1, n1, l1, f2_pack(xv.z, xv.z), f2_pack(xv.w, xv.w));
            }
        }
        if (fold_after(c0 + c + 1, B))
#pragma unroll
            for (int l = 0; l < S; ++l) df_acc2_renorm(acc[l]);
    }
}

// One block's units into acc; blk counts the group's blocks (its stage-value
// slot); false on a timeout.
template <int S, int B, bool XF, int CK, int NU, int R, int GO, int PW, class ACC>
__device__ __forceinline__ bool tp_block(ACC (&acc)[S], const unsigned char *gr, unsigned long long *fb,
                                         unsigned long long *eb, int &used, int blk, int a, int *err,
                                         volatile int *abort_flag) {
    using SH = TpShape<S, B, CK, NU, R, GO, PW>;
    constexpr int NCH = SH::UPB;
    constexpr int LAST = B - (NCH - 1) * CK;
    const float *X = reinterpret_cast<const float *>(gr + NU * SH::UNIT + (blk % SH::NX) * SH::XSLOT);
    // one copy of the unit's code (not unrolled over the chunks: the
    // unrolled form overflows the instruction cache)
#pragma unroll 1
    for (int ch = 0; ch < NCH; ++ch) {
        const int q = used % NU;
        if (!mbar_wait(fb + q, (unsigned)(used / NU) & 1u)) {
            atomicOr(err, IRK_DEV_ERR_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
        const unsigned char *unit = gr + q * SH::UNIT;
        const int c0 = ch * CK;
        if constexpr (R == 1) {
            if (LAST == CK || ch < NCH - 1)
                tp_consume<S, B, XF, CK>(acc, unit, X, c0, a);
            else
                tp_consume<S, B, XF, LAST>(acc, unit, X, c0, a);
        } else {
            if (LAST == CK || ch < NCH - 1)
                tp_consume2<S, B, XF, CK>(acc, unit, X, c0, a);
            else
                tp_consume2<S, B, XF, LAST>(acc, unit, X, c0, a);
        }
        mbar_arrive(eb + q);
        ++used;
    }
    return true;
}

// R = 2: a consumer thread owns rows a and a + 1 of its group's element row,
// their accumulators in packed two-lane instructions (df_acc2).
template <int S, int B, bool XF, int CK, int NU, int R, int GO = 0, int PW = 1, int MB = 0>
__global__ void __launch_bounds__(TpShape<S, B, CK, NU, R, GO, PW>::THREADS,
                                  MB > 0 ? MB
                                  : R == 2 ? 2
                                  : S <= 3 ? (XF ? 2048 : 1536) / TpShape<S, B, CK, NU, R, GO, PW>::THREADS
                                           : 1)
    k_matvec_tp(MatvecParams P, int *err) {
    using SH = TpShape<S, B, CK, NU, R, GO, PW>;
    using ACC = typename std::conditional<R == 1, df_acc, df_acc2>::type;
    constexpr int G = SH::G;
    constexpr long long BB = (long long)B * B, SB = (long long)S * B;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem_raw);  // [G][NU]
    unsigned long long *empty = full + G * NU;                                   // [G][NU]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem_raw + 2 * NU * G * 8);
    unsigned char *ring = smem_raw + SH::HEADER;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int q = 0; q < G * NU; ++q) {
            mbar_init_n(full + q, 1);
            mbar_init_n(empty + q, SH::BT);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int rstride = gridDim.x * G;  // T < 2^31
    if (tid >= SH::CONS) {
        // producer: lane g streams group g's units (one thread per group: a
        // single thread serving every group in turn with non-blocking tests
        // measured slower, 0.29 -> 0.33 ms on the 20000-triangle workload)
        const int lane = (tid - SH::CONS) & 31;
        const int g = ((tid - SH::CONS) >> 5) * SH::GPW + lane;
        if (lane >= SH::GPW || g >= G) return;
        unsigned long long *fb = full + g * NU, *eb = empty + g * NU;
        unsigned char *gr = ring + g * SH::GROUP;
        int issued = 0, nblk = 0;
        bool ok = true;
        // the pattern entries of the next row and block are loaded one row
        // and one block ahead, so that no copy waits on their latency
        int i = blockIdx.x * G + g;
        int p0 = 0, p1 = 0;
        if (i < P.T) {
            p0 = P.rp[i];
            p1 = P.rp[i + 1];
        }
        for (; i < P.T && ok; i += rstride) {
            const int in = i + rstride;
            int n0 = 0, n1 = 0;
            if (in < P.T) {
                n0 = P.rp[in];
                n1 = P.rp[in + 1];
            }
            const int pend = P.form != IRK_FORM_JACOBIAN ? p1 : p1 - 1;  // p == p1: the mass block
            int cnext = p0 < p1 ? P.ci[p0] : i;
            for (int p = p0; p <= pend && ok; ++p, ++nblk) {
                const int col = cnext;
                if (p + 1 < p1) cnext = P.ci[p + 1];
                const vec8 *blk = p < p1 ? P.J + (long long)p * BB : P.M + (long long)i * BB;
                const vec8 *xs = P.x + (long long)(p < p1 ? col : i) * SB;
                for (int c0 = 0; c0 < B; c0 += CK) {
                    const int nc = B - c0 < CK ? B - c0 : CK;
                    const int q = issued % NU;
                    if (issued >= NU && !mbar_wait(eb + q, (unsigned)((issued / NU) - 1) & 1u)) {
                        atomicOr(err, IRK_DEV_ERR_TIMEOUT);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    const unsigned jb = (unsigned)(nc * B * 8);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (c0 == 0) {
                        mbar_expect_arrive(fb + q, jb + (unsigned)SH::XSLOT);
                        tma_load_1d(gr + NU * SH::UNIT + (nblk % SH::NX) * SH::XSLOT, xs, (unsigned)SH::XSLOT, fb + q);
                    } else {
                        mbar_expect_arrive(fb + q, jb);
                    }
                    tma_load_1d(gr + q * SH::UNIT, blk + (long long)c0 * B, jb, fb + q);
                    ++issued;
                }
            }
            p0 = n0;
            p1 = n1;
        }
        // no copy into this CTA's shared memory may be in flight when it exits
        for (int u = issued > NU ? issued - NU : 0; u < issued; ++u) mbar_wait(fb + u % NU, (unsigned)(u / NU) & 1u);
        return;
    }
    const int g = tid / SH::BT, a = (tid - g * SH::BT) * R;
    if (g >= G) return;  // lanes past the last group
    unsigned long long *fb = full + g * NU, *eb = empty + g * NU;
    const unsigned char *gr = ring + g * SH::GROUP;
    int used = 0, nblk = 0;
    int i = blockIdx.x * G + g;
    int nb = i < P.T ? P.rp[i + 1] - P.rp[i] : 0;  // blocks of the row (the next row's: loaded a row ahead)
    for (; i < P.T; i += rstride) {
        const int in = i + rstride;
        const int nbn = in < P.T ? P.rp[in + 1] - P.rp[in] : 0;
        ACC t[S], z[S];
#pragma unroll
        for (int l = 0; l < S; ++l) {
            if constexpr (R == 1) {
                t[l] = df_acc_zero();
                z[l] = df_acc_zero();
            } else {
                t[l] = df_acc2_zero();
                z[l] = df_acc2_zero();
            }
        }
        for (int p = 0; p < nb; ++p)
            if (!tp_block<S, B, XF, CK, NU, R, GO, PW>(t, gr, fb, eb, used, nblk++, a, err, abort_flag)) return;
        if (P.form != IRK_FORM_JACOBIAN &&
            !tp_block<S, B, XF, CK, NU, R, GO, PW>(z, gr, fb, eb, used, nblk++, a, err, abort_flag))
            return;
        if constexpr (R == 1) {
            store_row<ArDF, S>(P, i, a, t, z);
        } else {
            df_acc t0[S], t1[S], z0[S], z1[S];
#pragma unroll
            for (int l = 0; l < S; ++l) {
                df_acc2_split(t[l], t0[l], t1[l]);
                df_acc2_split(z[l], z0[l], z1[l]);
            }
            store_row<ArDF, S>(P, i, a, t0, z0);
            store_row<ArDF, S>(P, i, a + 1, t1, z1);
        }
        nb = nbn;
    }
}

// k_matvec_tp with the element rows handed out at run time: each producer
// lane takes its group's next row from a global counter (zeroed by the
// launcher; one row ahead of the one it streams), so that every group keeps
// working until the rows run
// out instead of a fixed share of rows leaving a tail of groups with one row
// more than the others.  The producer writes each row's index and block
// count into a two-entry table of its group before the row's first unit; the
// consumers read it after that unit's "full" barrier (whose completion orders
// the write before their read), and a row index of -1, published with a
// "full" arrival that carries no copy, ends the group.  The table entry of a
// row is rewritten two rows later, by which time its consumers have moved on
// (a row spans more units than the ring holds).  Same accumulation order as
// every other variant; waits bounded as in k_matvec_tp.
template <int S, int B, bool XF, int CK, int NU, int R, int GO, int MB>
__global__ void __launch_bounds__(TpShape<S, B, CK, NU, R, GO, 1>::THREADS, MB)
    k_matvec_tpd(MatvecParams P, int *err) {
    using SH = TpShape<S, B, CK, NU, R, GO, 1>;
    using ACC = typename std::conditional<R == 1, df_acc, df_acc2>::type;
    constexpr int G = SH::G;
    constexpr long long BB = (long long)B * B, SB = (long long)S * B;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem_raw);  // [G][NU]
    unsigned long long *empty = full + G * NU;                                   // [G][NU]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem_raw + 2 * NU * G * 8);
    __shared__ int2 s_row[G][2];  // (row, J blocks) of a group's rows, by row ordinal parity
    unsigned char *ring = smem_raw + SH::HEADER;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int q = 0; q < G * NU; ++q) {
            mbar_init_n(full + q, 1);
            mbar_init_n(empty + q, SH::BT);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid >= SH::CONS) {
        const int g = tid - SH::CONS;
        if (g >= G) return;
        unsigned long long *fb = full + g * NU, *eb = empty + g * NU;
        unsigned char *gr = ring + g * SH::GROUP;
        int issued = 0, nblk = 0, nrow = 0, qend = -1;
        bool ok = true;
        int i = atomicAdd(P.rowctr, 1);
        int p0 = 0, p1 = 0;
        if (i < P.T) {
            p0 = P.rp[i];
            p1 = P.rp[i + 1];
        }
        while (ok) {
            // the slot of the row's first unit (or of the end marker)
            const int q0 = issued % NU;
            if (issued >= NU && !mbar_wait(eb + q0, (unsigned)((issued / NU) - 1) & 1u)) {
                atomicOr(err, IRK_DEV_ERR_TIMEOUT);
                *abort_flag = 1;
                break;
            }
            if (i >= P.T) {  // no rows left: end marker, a "full" arrival without a copy
                s_row[g][nrow & 1] = make_int2(-1, 0);
                mbar_arrive(fb + q0);
                qend = q0;
                break;
            }
            s_row[g][nrow & 1] = make_int2(i, p1 - p0);
            const int in = atomicAdd(P.rowctr, 1);  // the next row, consumed after this one
            const int pend = P.form != IRK_FORM_JACOBIAN ? p1 : p1 - 1;  // p == p1: the mass block
            int cnext = p0 < p1 ? P.ci[p0] : i;
            for (int p = p0; p <= pend && ok; ++p, ++nblk) {
                const int col = cnext;
                if (p + 1 < p1) cnext = P.ci[p + 1];
                const vec8 *blk = p < p1 ? P.J + (long long)p * BB : P.M + (long long)i * BB;
                const vec8 *xs = P.x + (long long)(p < p1 ? col : i) * SB;
                for (int c0 = 0; c0 < B; c0 += CK) {
                    const int nc = B - c0 < CK ? B - c0 : CK;
                    const int q = issued % NU;
                    // the first unit's slot was waited for above
                    if (!(p == p0 && c0 == 0) && issued >= NU &&
                        !mbar_wait(eb + q, (unsigned)((issued / NU) - 1) & 1u)) {
                        atomicOr(err, IRK_DEV_ERR_TIMEOUT);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    const unsigned jb = (unsigned)(nc * B * 8);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (c0 == 0) {
                        mbar_expect_arrive(fb + q, jb + (unsigned)SH::XSLOT);
                        tma_load_1d(gr + NU * SH::UNIT + (nblk % SH::NX) * SH::XSLOT, xs, (unsigned)SH::XSLOT, fb + q);
                    } else {
                        mbar_expect_arrive(fb + q, jb);
                    }
                    tma_load_1d(gr + q * SH::UNIT, blk + (long long)c0 * B, jb, fb + q);
                    ++issued;
                }
            }
            ++nrow;
            i = in;
            if (i < P.T) {
                p0 = P.rp[i];
                p1 = P.rp[i + 1];
            }
        }
        // no copy into this CTA's shared memory may be in flight when it
        // exits; the end marker completed one more phase of its slot, whose
        // earlier copy had landed before the marker was sent
        for (int u = issued > NU ? issued - NU : 0; u < issued; ++u)
            mbar_wait(fb + u % NU, ((unsigned)(u / NU) + (u % NU == qend ? 1u : 0u)) & 1u);
        return;
    }
    const int g = tid / SH::BT, a = (tid - g * SH::BT) * R;
    if (g >= G) return;
    unsigned long long *fb = full + g * NU, *eb = empty + g * NU;
    const unsigned char *gr = ring + g * SH::GROUP;
    int used = 0, nblk = 0;
    for (int nrow = 0;; ++nrow) {
        const int q0 = used % NU;
        if (!mbar_wait(fb + q0, (unsigned)(used / NU) & 1u)) {
            atomicOr(err, IRK_DEV_ERR_TIMEOUT);
            *abort_flag = 1;
            return;
        }
        const int2 row = s_row[g][nrow & 1];
        if (row.x < 0) return;
        const int i = row.x, nb = row.y;
        ACC t[S], z[S];
#pragma unroll
        for (int l = 0; l < S; ++l) {
            if constexpr (R == 1) {
                t[l] = df_acc_zero();
                z[l] = df_acc_zero();
            } else {
                t[l] = df_acc2_zero();
                z[l] = df_acc2_zero();
            }
        }
        for (int p = 0; p < nb; ++p)
            if (!tp_block<S, B, XF, CK, NU, R, GO, 1>(t, gr, fb, eb, used, nblk++, a, err, abort_flag)) return;
        if (P.form != IRK_FORM_JACOBIAN &&
            !tp_block<S, B, XF, CK, NU, R, GO, 1>(z, gr, fb, eb, used, nblk++, a, err, abort_flag))
            return;
        if constexpr (R == 1) {
            store_row<ArDF, S>(P, i, a, t, z);
        } else {
            df_acc t0[S], t1[S], z0[S], z1[S];
#pragma unroll
            for (int l = 0; l < S; ++l) {
                df_acc2_split(t[l], t0[l], t1[l]);
                df_acc2_split(z[l], z0[l], z1[l]);
            }
            store_row<ArDF, S>(P, i, a, t0, z0);
            store_row<ArDF, S>(P, i, a + 1, t1, z1);
        }
    }
}

template <int S, int B, int CK, int NU, int R, int GO, int MB>
bool run_matvec_tpd(const MatvecParams &P, int *err, cudaStream_t st) {
    if (P.m != B || !P.rowctr || P.form == IRK_FORM_JACOBIAN) return false;
    using SH = TpShape<S, B, CK, NU, R, GO, 1>;
    const void *kern = P.xf32 ? (const void *)k_matvec_tpd<S, B, true, CK, NU, R, GO, MB>
                              : (const void *)k_matvec_tpd<S, B, false, CK, NU, R, GO, MB>;
    if (irk_allow_max_smem(kern)) return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH::THREADS, SH::SMEM) != cudaSuccess ||
        per_sm <= 0)
        return false;
    const long long need = (P.T + SH::G - 1) / SH::G;
    const long long grid = std::max(1LL, std::min<long long>(need, (long long)dev_limits().sms * per_sm));
    if (cudaMemsetAsync(P.rowctr, 0, sizeof(int), st) != cudaSuccess) return false;
    if (P.xf32)
        k_matvec_tpd<S, B, true, CK, NU, R, GO, MB><<<(int)grid, SH::THREADS, SH::SMEM, st>>>(P, err);
    else
        k_matvec_tpd<S, B, false, CK, NU, R, GO, MB><<<(int)grid, SH::THREADS, SH::SMEM, st>>>(P, err);
    return true;
}

template <int S, int CK, int NU, int R, int GO, int MB>
bool run_matvec_tpd_any(const MatvecParams &P, int *err, cudaStream_t st) {
    return run_matvec_tpd<S, 40, CK, NU, R, GO, MB>(P, err, st) ||
           run_matvec_tpd<S, 50, CK, NU, R, GO, MB>(P, err, st) ||
           run_matvec_tpd<S, 24, CK, NU, R, GO, MB>(P, err, st) ||
           run_matvec_tpd<S, 20, CK, NU, R, GO, MB>(P, err, st) ||
           run_matvec_tpd<S, 12, CK, NU, R, GO, MB>(P, err, st);
}

template <int S, int B, int CK, int NU, int R, int GO = 0, int PW = 1, int MB = 0>
bool run_matvec_tp(const MatvecParams &P, int *err, cudaStream_t st) {
    if (P.m != B) return false;
    using SH = TpShape<S, B, CK, NU, R, GO, PW>;
    static_assert(B % 2 == 0, "bulk copies need 16-byte multiples");
    const void *kern = P.xf32 ? (const void *)k_matvec_tp<S, B, true, CK, NU, R, GO, PW, MB>
                              : (const void *)k_matvec_tp<S, B, false, CK, NU, R, GO, PW, MB>;
    if (irk_allow_max_smem(kern)) return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH::THREADS, SH::SMEM) != cudaSuccess ||
        per_sm <= 0)
        return false;
    const long long need = (P.T + SH::G - 1) / SH::G;
    const long long grid = std::max(1LL, std::min<long long>(need, (long long)dev_limits().sms * per_sm));
    if (P.xf32)
        k_matvec_tp<S, B, true, CK, NU, R, GO, PW, MB><<<(int)grid, SH::THREADS, SH::SMEM, st>>>(P, err);
    else
        k_matvec_tp<S, B, false, CK, NU, R, GO, PW, MB><<<(int)grid, SH::THREADS, SH::SMEM, st>>>(P, err);
    return true;
}

template <int S, int CK, int NU, int R = 1, int GO = 0, int MB = 0>
bool run_matvec_tp_any(const MatvecParams &P, int *err, cudaStream_t st) {
    return run_matvec_tp<S, 40, CK, NU, R, GO, 1, MB>(P, err, st) ||
           run_matvec_tp<S, 50, CK, NU, R, GO, 1, MB>(P, err, st) ||
           run_matvec_tp<S, 24, CK, NU, R, GO, 1, MB>(P, err, st) ||
           run_matvec_tp<S, 20, CK, NU, R, GO, 1, MB>(P, err, st) ||
           run_matvec_tp<S, 12, CK, NU, R, GO, 1, MB>(P, err, st);
}

template <int S>
bool run_tp_s(const MatvecParams &P, int form, int *err, cudaStream_t st) {
    switch (form) {
        case 5: return run_matvec_tp_any<S, 8, 4>(P, err, st);
        case 6: return run_matvec_tp_any<S, 16, 2>(P, err, st);
        case 7: return run_matvec_tp_any<S, 8, 3>(P, err, st);
        case 8: return run_matvec_tp_any<S, 8, 3, 2, 128>(P, err, st);
        case 9: return run_matvec_tp_any<S, 8, 2, 2, 128>(P, err, st);
        case 10: return run_matvec_tp_any<S, 8, 2, 2, 128, 5>(P, err, st);
        case 11: return run_matvec_tpd_any<S, 8, 2, 2, 128, 5>(P, err, st);
        case 12: return run_matvec_tpd_any<S, 8, 2, 2, 128, 4>(P, err, st);
        default: return false;
    }
}

}  // namespace

bool run_matvec_tp_form(const MatvecParams &P, int s, int form, int *err, cudaStream_t st) {
    if ((((uintptr_t)P.x | (uintptr_t)P.J | (uintptr_t)P.M) & 15) != 0) return false;
    switch (s) {
        case 2: return run_tp_s<2>(P, form, err, st);
        case 3: return run_tp_s<3>(P, form, err, st);
        case 4: return run_tp_s<4>(P, form, err, st);
        default: return false;
    }
}

}  // namespace irk_mv
