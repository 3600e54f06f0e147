// planes_batched.cu -- the planes forward transform of many volumes of
// different sizes in one persistent launch.
//
// Work items are runs of consecutive unit-tiles (a unit of a fused pass, see
// planes_fused.cu, with one of its displacement tiles; a unit's tiles are
// consecutive) of every fused pass of every volume and dodecant; the run
// length is a per-(size, pass) setting (drt3d_batch_set_item_tiles).  Items
// are numbered pass-major: all first-pass items of all volumes, then all
// second-pass items, ...; within a (pass, volume) segment item i belongs to
// dodecant slot i / (items per slot).  Resident
// CTAs (two per SM) take items from an atomic counter.  An item of pass p > 0
// reads the intermediate written by every pass p-1 item of its (volume,
// dodecant); those items were all handed out before it, to CTAs that are
// running, so the item waits for their completion counter -- a bounded wait:
// after the time limit it records DRT3D_ERR_TIMEOUT in the status word, sets
// an abort flag that ends all other waits, and skips its work.
//
// One call is one memset of the counters and one kernel launch on the
// caller's stream, so it can be captured in a CUDA graph.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "fused_cta.cuh"

namespace drt3d {

constexpr int kBatchMaxPass = 4;
constexpr int kBatchMaxStreams = 8;

struct BatchVol {
    CUtensorMap tmap[kBatchMaxPass];  // TMA view of each pass's 16-bit input (passes that stage it)
    FusedLaunch pass[kBatchMaxPass];
    int tma[kBatchMaxPass];           // pass stages its input through tmap[p]
    int npass;
    int G[kBatchMaxPass];
    int in_kind[kBatchMaxPass], out_kind[kBatchMaxPass];
    unsigned ctas[kBatchMaxPass];  // items per dodecant slot
    unsigned tpi[kBatchMaxPass];   // unit-tiles per item (consecutive in unit-major order)
    unsigned cps[kBatchMaxPass];   // unit-tiles per dodecant slot
};

struct BatchArgs {
    const BatchVol* vols;
    const unsigned* seg_start;  // nseg + 1 entries
    const int* seg_vol;
    const int* seg_pass;
    int nseg;
    unsigned nitems;
    unsigned* next;     // work counter
    unsigned* abort;    // set once a wait gives up
    unsigned* done;     // [vol][12][kBatchMaxPass] completed items
    int* status;
    unsigned long long wait_ns;
    int withhold_vol, withhold_slot;  // test hook: this (vol, slot) never signals pass 0
};

namespace {

using namespace fused;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 only: wait until *ctr >= target.  Returns false when it gives up.
__device__ bool wait_counter(const BatchArgs& A, const unsigned* ctr, unsigned target) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (*(volatile const unsigned*)ctr >= target) {
            __threadfence();
            return true;
        }
        if (*(volatile const unsigned*)A.abort) return false;
        if (global_ns() - t0 > A.wait_ns) {
            atomicCAS(A.status, 0, (int)DRT3D_ERR_TIMEOUT);
            atomicExch(A.abort, 1u);
            return false;
        }
        __nanosleep(256);
    }
}

// The item's pass header and dodecant slot are copied into registers: read
// through a global pointer, the compiler would have to reload them after every
// store (it cannot prove the output buffers do not alias the tables).
template <typename TIn, typename TOut, typename TS, int G, bool INGEST, bool TMA = false>
__device__ __forceinline__ void run_g(const FusedLaunch& Lg, int slot, unsigned item, unsigned tpi, unsigned cps,
                                      unsigned char* smem, const CUtensorMap* tmap = nullptr,
                                      uint64_t* mbar = nullptr, int* status = nullptr) {
    FusedLaunch L;
    L.N = Lg.N;
    L.n = Lg.n;
    L.m0 = Lg.m0;
    L.gin = Lg.gin;
    L.gout = Lg.gout;
    L.dmax = Lg.dmax;
    L.V = Lg.V;
    L.ntiles = Lg.ntiles;
    L.ctas = Lg.ctas;
    L.vec_store = Lg.vec_store;
    L.prefetch_ahead = 0;  // launch order is not item order here (and the prefetch is compiled out)
    L.reverse_slots = 0;
    L.status = status;
    L.global_layout = 0;
    const FusedSlot sp = Lg.slot[slot];
    // one item = `tpi` consecutive unit-tiles (unit-major: a unit's tiles are consecutive)
    const unsigned c0 = item * tpi, c1 = min(c0 + tpi, cps);
    // The staged rows were written by other CTAs through the generic proxy
    // (made visible to this one by the dependency wait): one proxy fence per
    // thread orders them before all of this item's TMA reads.
    if constexpr (TMA) tma::fence_proxy_async_global();
    for (unsigned c = c0; c < c1; ++c) {
        if (c > c0) __syncthreads();  // the previous tile's phase 2 is done with shared memory
        if constexpr (TMA)
            fused_cta<TIn, TOut, uint32_t, TS, G, false, false, true, false>(L, sp, c, smem, tmap, slot, mbar);
        else if constexpr (INGEST && G == 4 && std::is_same<TIn, uint8_t>::value && std::is_same<TS, uint16_t>::value)
            fused_cta_u8x2<TOut, G>(L, sp, c, smem);  // 16-bit sums: two groups per register
        else
            fused_cta<TIn, TOut, uint32_t, TS, G, INGEST, true, false, false>(L, sp, c, smem);
    }
}

template <typename TIn, typename TOut, typename TS, bool INGEST>
__device__ __forceinline__ void run_kind(const FusedLaunch& L, int G, int slot, unsigned item, unsigned tpi,
                                         unsigned cps, unsigned char* smem) {
    switch (G) {
    case 2: run_g<TIn, TOut, TS, 2, INGEST>(L, slot, item, tpi, cps, smem); break;
    case 3: run_g<TIn, TOut, TS, 3, INGEST>(L, slot, item, tpi, cps, smem); break;
    default: run_g<TIn, TOut, TS, 4, INGEST>(L, slot, item, tpi, cps, smem); break;
    }
}

__global__ void __launch_bounds__(256, 2) planes_batched(const __grid_constant__ BatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[16];
    // 128-byte aligned for TMA destinations
    unsigned char* smem = smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ unsigned s_item, s_next;
    __shared__ int s_go, s_seg;
    // The next item is claimed while the current one runs, hiding the
    // atomic's round trip.  A CTA's items only increase, so its segment is
    // found by advancing a cursor (amortised O(1)).
    int seg = 0;  // thread 0's cursor
    if (threadIdx.x == 0) s_next = atomicAdd(A.next, 1u);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned it = s_next;
            s_item = it;
            if (it < A.nitems) {
                s_next = atomicAdd(A.next, 1u);
                while (__ldg(A.seg_start + seg + 1) <= it) ++seg;
                s_seg = seg;
            }
        }
        __syncthreads();
        const unsigned item = s_item;
        if (item >= A.nitems) return;
        const int lo = s_seg;
        const int v = __ldg(A.seg_vol + lo), p = __ldg(A.seg_pass + lo);
        const BatchVol& B = A.vols[v];
        const unsigned local = item - __ldg(A.seg_start + lo);
        const unsigned ctas_p = B.ctas[p];
        const int slot = (int)(local / ctas_p);
        const unsigned cta = local - (unsigned)slot * ctas_p;
        unsigned* done = A.done + ((size_t)v * kMaxSlots + slot) * kBatchMaxPass;
        if (p > 0) {
            if (threadIdx.x == 0) s_go = wait_counter(A, done + (p - 1), B.ctas[p - 1]) ? 1 : 0;
            __syncthreads();
            if (!s_go) continue;
        }
        const FusedLaunch& L = B.pass[p];
        const int G = B.G[p];
        const int ik = B.in_kind[p], ok = B.out_kind[p];
        const unsigned tpi = B.tpi[p], cps = B.cps[p];
        if (p == 0) {
            if (ok == (int)ElemKind::U16) run_kind<uint8_t, uint16_t, uint16_t, true>(L, G, slot, cta, tpi, cps, smem);
            else run_kind<uint8_t, uint32_t, uint16_t, true>(L, G, slot, cta, tpi, cps, smem);
        } else if (B.tma[p]) {
            // 16-bit input staged by TMA (G >= 3)
            const CUtensorMap* tm = &B.tmap[p];
            if (G == 4) {
                if (ok == (int)ElemKind::U16)
                    run_g<uint16_t, uint16_t, uint32_t, 4, false, true>(L, slot, cta, tpi, cps, smem, tm, mbar,
                                                                        A.status);
                else
                    run_g<uint16_t, uint32_t, uint32_t, 4, false, true>(L, slot, cta, tpi, cps, smem, tm, mbar,
                                                                        A.status);
            } else {
                if (ok == (int)ElemKind::U16)
                    run_g<uint16_t, uint16_t, uint32_t, 3, false, true>(L, slot, cta, tpi, cps, smem, tm, mbar,
                                                                        A.status);
                else
                    run_g<uint16_t, uint32_t, uint32_t, 3, false, true>(L, slot, cta, tpi, cps, smem, tm, mbar,
                                                                        A.status);
            }
        } else if (ik == (int)ElemKind::U16) {
            if (ok == (int)ElemKind::U16) run_kind<uint16_t, uint16_t, uint32_t, false>(L, G, slot, cta, tpi, cps, smem);
            else run_kind<uint16_t, uint32_t, uint32_t, false>(L, G, slot, cta, tpi, cps, smem);
        } else {
            run_kind<uint32_t, uint32_t, uint32_t, false>(L, G, slot, cta, tpi, cps, smem);
        }
        // Signal completion only where a later pass depends on it.
        if (p + 1 < B.npass) {
            __syncthreads();
            if (threadIdx.x == 0 && !(p == 0 && v == A.withhold_vol && slot == A.withhold_slot)) {
                __threadfence();
                atomicAdd(done + p, 1u);
            }
        }
    }
}

size_t batched_smem_bytes() { return ((size_t)(1 << 8) * fused_ws<4>() + fused_pad<4>()) * sizeof(uint32_t) + 128; }

}  // namespace

// Opt the kernel into its shared-memory size once per device (done at bind,
// so a launch inside stream capture issues only stream work).
cudaError_t batched_prepare(int device) {
    static DeviceOnce done;
    if (done.done(device)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(planes_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batched_smem_bytes());
    if (e == cudaSuccess) done.mark(device);
    return e;
}

cudaError_t launch_planes_batched(const BatchArgs& A, int grid, cudaStream_t s) {
    planes_batched<<<grid, 256, batched_smem_bytes(), s>>>(A);
    return cudaGetLastError();
}

int batched_grid(int device) {
    if (batched_prepare(device) != cudaSuccess) return 0;
    int sms = 0, per = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, planes_batched, 256, batched_smem_bytes()) != cudaSuccess)
        return 0;
    return sms * std::max(per, 1);
}

}  // namespace drt3d

using namespace drt3d;

struct drt3d_batch_plan {
    int count = 0;
    std::vector<int> Ns;
    drt3d_dtype dtype = DRT3D_U8;
    int device = 0;
    int* d_status = nullptr;
    std::vector<FusedSchedule> sched;  // per volume
    // Work-item size of the persistent launch per volume size: unit-tiles per
    // item of each pass (0 or absent: the default of item_tiles_default).
    std::map<int, std::vector<int>> item_tiles;
    // bound state
    bool bound = false;
    BatchVol* d_vols = nullptr;
    unsigned* d_seg_start = nullptr;
    int* d_seg_vol = nullptr;
    int* d_seg_pass = nullptr;
    unsigned* d_counters = nullptr;  // next, abort, done[count][12][kBatchMaxPass]
    size_t counters_bytes = 0;
    int nseg = 0;
    unsigned nitems = 0;
    int grid = 0;
    unsigned long long wait_ns = 2000000000ull;
    int withhold_vol = -1, withhold_slot = -1;
    // Mode 1: each volume's passes as ordinary launches, volumes spread over
    // internal streams (forked from and joined back into the caller's).
    int mode = 0;
    int nstreams = 0;
    cudaStream_t streams[kBatchMaxStreams] = {};
    cudaEvent_t fork = nullptr, join[kBatchMaxStreams] = {};
    std::vector<BatchVol> hvols;       // host copy of the bound descriptors
    std::vector<int> vol_stream;       // stream of each volume
    std::vector<size_t> vol_slot_stride;
};

namespace {

void free_streams(drt3d_batch_plan* B) {
    for (int i = 0; i < B->nstreams; ++i) {
        if (B->streams[i]) cudaStreamDestroy(B->streams[i]);
        if (B->join[i]) cudaEventDestroy(B->join[i]);
        B->streams[i] = nullptr;
        B->join[i] = nullptr;
    }
    if (B->fork) cudaEventDestroy(B->fork);
    B->fork = nullptr;
    B->nstreams = 0;
}

// Volumes to streams, largest first onto the least loaded stream (work ~ N^3).
void assign_streams(drt3d_batch_plan* B) {
    const int k = std::max(1, B->nstreams);
    std::vector<int> order(B->count);
    for (int v = 0; v < B->count; ++v) order[v] = v;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B->Ns[a] > B->Ns[b]; });
    std::vector<double> load(k, 0.0);
    B->vol_stream.assign(B->count, 0);
    for (int v : order) {
        const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        B->vol_stream[v] = s;
        load[s] += (double)B->Ns[v] * B->Ns[v] * B->Ns[v];
    }
}

void free_bound(drt3d_batch_plan* B) {
    cudaFree(B->d_vols);
    cudaFree(B->d_seg_start);
    cudaFree(B->d_seg_vol);
    cudaFree(B->d_seg_pass);
    cudaFree(B->d_counters);
    B->d_vols = nullptr;
    B->d_seg_start = nullptr;
    B->d_seg_vol = nullptr;
    B->d_seg_pass = nullptr;
    B->d_counters = nullptr;
    B->bound = false;
}

size_t vol_ws_bytes(const FusedSchedule& S) { return S.npass > 1 ? (size_t)kMaxSlots * 2 * S.buf_bytes : 0; }

// Default work-item size in unit-tiles: 8 tiles at G = 4 (measured best among
// 1..48 on the N = 256 and N = 128 batches: shorter items pay their claim,
// dependency check and completion signal too often, longer ones balance
// worse), otherwise `upi` whole units.
unsigned item_tiles_default(int G, unsigned upi, int ntiles) { return G >= 4 ? 8u : upi * (unsigned)ntiles; }

}  // namespace

extern "C" {

drt3d_status drt3d_batch_plan_create(drt3d_batch_plan** plan, int count, const int* Ns, drt3d_dtype dtype,
                                     unsigned flags) {
    if (!plan) return DRT3D_ERR_INVALID_ARG;
    *plan = nullptr;
    if (count <= 0 || !Ns || flags != 0) return DRT3D_ERR_INVALID_ARG;
    if (dtype != DRT3D_U8) return DRT3D_ERR_DTYPE;
    for (int i = 0; i < count; ++i)
        if (Ns[i] < 16 || Ns[i] > 256 || (Ns[i] & (Ns[i] - 1))) return DRT3D_ERR_SIZE;
    drt3d_batch_plan* B = new (std::nothrow) drt3d_batch_plan();
    if (!B) return DRT3D_ERR_NO_MEMORY;
    B->count = count;
    B->Ns.assign(Ns, Ns + count);
    B->dtype = dtype;
    if (cudaGetDevice(&B->device) != cudaSuccess) { delete B; return DRT3D_ERR_CUDA; }
    if (cudaMalloc(&B->d_status, sizeof(int)) != cudaSuccess) { delete B; return DRT3D_ERR_NO_MEMORY; }
    cudaMemset(B->d_status, 0, sizeof(int));
    for (int i = 0; i < count; ++i) B->sched.push_back(make_fused_schedule(Ns[i], dtype));
    *plan = B;
    return DRT3D_OK;
}

drt3d_status drt3d_batch_plan_destroy(drt3d_batch_plan* B) {
    if (!B) return DRT3D_OK;
    free_bound(B);
    free_streams(B);
    cudaFree(B->d_status);
    delete B;
    return DRT3D_OK;
}

drt3d_status drt3d_batch_set_schedule(drt3d_batch_plan* B, int N, int ngroups, const int* G) {
    if (!B || !G) return DRT3D_ERR_INVALID_ARG;
    if (ngroups < 1 || ngroups > kBatchMaxPass) return DRT3D_ERR_INVALID_ARG;
    int sum = 0;
    for (int g = 0; g < ngroups; ++g) {
        if (G[g] < 2 || G[g] > 4) return DRT3D_ERR_INVALID_ARG;
        sum += G[g];
    }
    if ((1 << sum) != N) return DRT3D_ERR_SIZE;
    FusedSchedule S;
    if (!make_fused_schedule_groups(N, B->dtype, ngroups, G, &S)) return DRT3D_ERR_INVALID_ARG;
    for (int i = 0; i < B->count; ++i)
        if (B->Ns[i] == N) B->sched[i] = S;
    B->item_tiles.erase(N);  // sized for the previous schedule's passes
    if (B->bound) free_bound(B);
    return DRT3D_OK;
}

drt3d_status drt3d_batch_set_item_tiles(drt3d_batch_plan* B, int N, int npass, const int* tiles) {
    if (!B || !tiles) return DRT3D_ERR_INVALID_ARG;
    const int i = (int)(std::find(B->Ns.begin(), B->Ns.end(), N) - B->Ns.begin());
    if (i == B->count) return DRT3D_ERR_SIZE;  // no volume of this size in the batch
    if (npass != B->sched[i].npass) return DRT3D_ERR_INVALID_ARG;
    for (int p = 0; p < npass; ++p)
        if (tiles[p] < 0) return DRT3D_ERR_INVALID_ARG;
    B->item_tiles[N].assign(tiles, tiles + npass);
    if (B->bound) free_bound(B);
    return DRT3D_OK;
}

drt3d_status drt3d_batch_workspace_bytes(const drt3d_batch_plan* B, size_t* bytes) {
    if (!B || !bytes) return DRT3D_ERR_INVALID_ARG;
    size_t t = 0;
    for (int i = 0; i < B->count; ++i) t += align_up(vol_ws_bytes(B->sched[i]), 256);
    *bytes = t;
    return DRT3D_OK;
}

drt3d_status drt3d_batch_bind(drt3d_batch_plan* B, const drt3d_vol_desc* descs, void* d_ws, size_t ws_bytes) {
    if (!B || !descs) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(B->device)) return DRT3D_ERR_INVALID_ARG;
    size_t need = 0;
    drt3d_batch_workspace_bytes(B, &need);
    if (need > 0 && (!d_ws || ws_bytes < need)) return DRT3D_ERR_WORKSPACE;
    for (int i = 0; i < B->count; ++i) {
        if (!descs[i].d_in || !descs[i].d_out) return DRT3D_ERR_INVALID_ARG;
        if (((uintptr_t)descs[i].d_in & 15) || ((uintptr_t)descs[i].d_out & 15)) return DRT3D_ERR_ALIGN;
    }
    if (((uintptr_t)d_ws & 15)) return DRT3D_ERR_ALIGN;
    free_bound(B);
    B->vol_slot_stride.clear();
    std::vector<BatchVol> vols(B->count);
    char* ws = static_cast<char*>(d_ws);
    int maxpass = 0;
    for (int v = 0; v < B->count; ++v) {
        const int N = B->Ns[v];
        const FusedSchedule& S = B->sched[v];
        BatchVol& bv = vols[v];
        std::memset(&bv, 0, sizeof(bv));
        bv.npass = S.npass;
        maxpass = std::max(maxpass, S.npass);
        const size_t buf = S.buf_bytes;
        const size_t out_block = (size_t)N * N * 3 * N * 4;
        for (int p = 0; p < S.npass; ++p) {
            const FusedPass& ps = S.pass[p];
            FusedLaunch& L = bv.pass[p];
            L.N = N;
            L.n = ilog2(N);
            L.dmax = 3 * N;
            L.m0 = ps.m0;
            L.gin = ps.in;
            L.gout = ps.out;
            L.V = fused_valid(ps.G);
            L.ntiles = (3 * N - ps.out.base + L.V - 1) / L.V;
            const long long per_axis = 1LL << (L.n - ps.G);
            L.ctas = per_axis * per_axis * L.ntiles;
            L.vec_store = (ps.out.pitch % 4 == 0) && (ps.out.base % 4 == 0) && (3 * N) % 4 == 0;
            for (int k = 0; k < 12; ++k) {
                char* bufA = ws + (size_t)k * 2 * buf;
                char* bufB = bufA + buf;
                FusedSlot& fs = L.slot[k];
                fs.map = dodecant_affine(N, k);
                fused_ingest_mode(N, fs.map, fs);
                fs.in = (p == 0) ? descs[v].d_in : ((p & 1) ? (const void*)bufA : (const void*)bufB);
                fs.out = ps.final_ ? (void*)(reinterpret_cast<char*>(descs[v].d_out) + (size_t)k * out_block)
                                   : ((p & 1) ? (void*)bufB : (void*)bufA);
            }
            bv.G[p] = ps.G;
            // (the persistent kernel stages 16-bit rows only)
            bv.tma[p] = fused_uses_tma(ps.G, ps.in_kind, ps.ingest) && ps.in_kind == ElemKind::U16 ? 1 : 0;
            if (bv.tma[p] && encode_fused_tmap(L, L.slot[0].in, 2 * buf, 12, 2, &bv.tmap[p]) != cudaSuccess)
                return DRT3D_ERR_CUDA;
            bv.in_kind[p] = (int)ps.in_kind;
            bv.out_kind[p] = (int)ps.out_kind;
            // Small units (2^G x 2^G rows) are grouped so that an item carries
            // at least 256 rows: its claim, dependency wait and barriers would
            // otherwise cost more than its work.
            bv.cps[p] = (unsigned)L.ctas;
            const unsigned upi = ps.G >= 4 ? 1u : (ps.G == 3 ? 4u : (ps.G == 2 ? 16u : 64u));
            const auto it = B->item_tiles.find(N);
            const int want = it != B->item_tiles.end() && p < (int)it->second.size() ? it->second[p] : 0;
            bv.tpi[p] = want > 0 ? std::min((unsigned)want, bv.cps[p]) : item_tiles_default(ps.G, upi, L.ntiles);
            bv.ctas[p] = (bv.cps[p] + bv.tpi[p] - 1) / bv.tpi[p];
        }
        B->vol_slot_stride.push_back(2 * buf);
        ws += align_up(vol_ws_bytes(S), 256);
    }
    B->hvols = vols;
    assign_streams(B);
    // pass-major segments
    std::vector<unsigned> seg_start;
    std::vector<int> seg_vol, seg_pass;
    unsigned n = 0;
    for (int p = 0; p < maxpass; ++p)
        for (int v = 0; v < B->count; ++v) {
            if (p >= vols[v].npass) continue;
            seg_start.push_back(n);
            seg_vol.push_back(v);
            seg_pass.push_back(p);
            n += vols[v].ctas[p] * 12u;
        }
    seg_start.push_back(n);
    B->nseg = (int)seg_vol.size();
    B->nitems = n;
    B->counters_bytes = (2 + (size_t)B->count * kMaxSlots * kBatchMaxPass) * sizeof(unsigned);
    bool ok = cudaMalloc(&B->d_vols, vols.size() * sizeof(BatchVol)) == cudaSuccess &&
              cudaMalloc(&B->d_seg_start, seg_start.size() * sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&B->d_seg_vol, seg_vol.size() * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&B->d_seg_pass, seg_pass.size() * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&B->d_counters, B->counters_bytes) == cudaSuccess;
    if (!ok) { free_bound(B); return DRT3D_ERR_NO_MEMORY; }
    ok = cudaMemcpy(B->d_vols, vols.data(), vols.size() * sizeof(BatchVol), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(B->d_seg_start, seg_start.data(), seg_start.size() * sizeof(unsigned),
                    cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(B->d_seg_vol, seg_vol.data(), seg_vol.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(B->d_seg_pass, seg_pass.data(), seg_pass.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) { free_bound(B); return DRT3D_ERR_CUDA; }
    B->grid = batched_grid(B->device);
    if (B->grid <= 0) { free_bound(B); return DRT3D_ERR_CUDA; }
    B->bound = true;
    return DRT3D_OK;
}

drt3d_status drt3d_batch_set_mode(drt3d_batch_plan* B, int mode, int nstreams) {
    if (!B || (mode != 0 && mode != 1)) return DRT3D_ERR_INVALID_ARG;
    if (mode == 1 && (nstreams < 1 || nstreams > kBatchMaxStreams)) return DRT3D_ERR_INVALID_ARG;
    free_streams(B);
    B->mode = mode;
    if (mode == 1) {
        for (int i = 0; i < nstreams; ++i) {
            if (cudaStreamCreateWithFlags(&B->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming) != cudaSuccess) {
                B->nstreams = i + 1;
                free_streams(B);
                B->mode = 0;
                return DRT3D_ERR_CUDA;
            }
        }
        B->nstreams = nstreams;
        if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) {
            free_streams(B);
            B->mode = 0;
            return DRT3D_ERR_CUDA;
        }
    }
    if (B->bound) assign_streams(B);
    return DRT3D_OK;
}

drt3d_status drt3d_planes_forward_batched(const drt3d_batch_plan* B, cudaStream_t stream) {
    if (!B || !B->bound) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(B->device)) return DRT3D_ERR_INVALID_ARG;
    if (B->mode == 1) {
        // pass-major over the volumes; a volume's passes stay on its stream
        if (cudaEventRecord(B->fork, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
        for (int i = 0; i < B->nstreams; ++i)
            if (cudaStreamWaitEvent(B->streams[i], B->fork, 0) != cudaSuccess) return DRT3D_ERR_CUDA;
        int maxpass = 0;
        for (const BatchVol& bv : B->hvols) maxpass = std::max(maxpass, bv.npass);
        for (int p = 0; p < maxpass; ++p)
            for (int v = 0; v < B->count; ++v) {
                const BatchVol& bv = B->hvols[v];
                if (p >= bv.npass) continue;
                FusedLaunch L = bv.pass[p];
                L.status = B->d_status;
                const cudaStream_t st = B->streams[B->vol_stream[v]];
                cudaError_t e;
                if (bv.tma[p])
                    e = launch_planes_fused_tma(L, bv.G[p], (ElemKind)bv.in_kind[p], (ElemKind)bv.out_kind[p],
                                                L.slot[0].in,
                                                B->vol_slot_stride[v], 12, st);
                else
                    e = launch_planes_fused(L, bv.G[p], (ElemKind)bv.in_kind[p], (ElemKind)bv.out_kind[p], p == 0,
                                            12, st);
                if (e != cudaSuccess) return DRT3D_ERR_CUDA;
            }
        for (int i = 0; i < B->nstreams; ++i) {
            if (cudaEventRecord(B->join[i], B->streams[i]) != cudaSuccess) return DRT3D_ERR_CUDA;
            if (cudaStreamWaitEvent(stream, B->join[i], 0) != cudaSuccess) return DRT3D_ERR_CUDA;
        }
        return DRT3D_OK;
    }
    if (cudaMemsetAsync(B->d_counters, 0, B->counters_bytes, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    BatchArgs A;
    A.vols = B->d_vols;
    A.seg_start = B->d_seg_start;
    A.seg_vol = B->d_seg_vol;
    A.seg_pass = B->d_seg_pass;
    A.nseg = B->nseg;
    A.nitems = B->nitems;
    A.next = B->d_counters;
    A.abort = B->d_counters + 1;
    A.done = B->d_counters + 2;
    A.status = B->d_status;
    A.wait_ns = B->wait_ns;
    A.withhold_vol = B->withhold_vol;
    A.withhold_slot = B->withhold_slot;
    if (launch_planes_batched(A, B->grid, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    return DRT3D_OK;
}

drt3d_status drt3d_batch_get_device_error(const drt3d_batch_plan* B, cudaStream_t stream) {
    if (!B) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(B->device)) return DRT3D_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    int h = 0;
    if (cudaMemcpy(&h, B->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DRT3D_ERR_CUDA;
    if (h != 0 && cudaMemset(B->d_status, 0, sizeof(int)) != cudaSuccess) return DRT3D_ERR_CUDA;
    return (drt3d_status)h;
}

drt3d_status drt3d_batch_set_wait_limit(drt3d_batch_plan* B, unsigned long long ns, int withhold_vol,
                                        int withhold_dodecant) {
    if (!B || ns == 0) return DRT3D_ERR_INVALID_ARG;
    B->wait_ns = ns;
    B->withhold_vol = withhold_vol;
    B->withhold_slot = withhold_dodecant;
    return DRT3D_OK;
}

}  // extern "C"
