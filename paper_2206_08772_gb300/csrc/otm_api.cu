// otm_api.cu -- the C ABI (include/otm.h): workspace layout, initialisation, the step driver
// (Algorithm 1 as a fixed kernel sequence on one stream) and state transfer.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include <new>

#include "otm_dev.cuh"

using namespace otm;

struct otm_handle {
    Dev D;
    otm_params P;
    cudaStream_t stream;
    void *ws;
    size_t ws_bytes;
    int32_t *scan_tmp;
    int64_t step;
    long long launches;
    int64_t n_eroded, n_removed, n_inserted;
    int64_t nn0, nm0;              // sizes at initialisation
    int64_t nn_cap;                // node array capacity (nn0 + max_insert)
    bool frozen;                   // topology frozen: steps keep their supports
    // adjoint
    void *adj_ws;
    bool adj_swap;
    // phase timing
    bool timing;
    struct Rec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    double phase_ms[OTM_N_PHASES];
    int64_t phase_n[OTM_N_PHASES];
};

// bracket one phase with events when timing is on
struct PhaseScope {
    otm_handle *h;
    int phase;
    cudaEvent_t a = nullptr, b = nullptr;
    PhaseScope(otm_handle *h_, int ph) : h(h_), phase(ph)
    {
        if (h->timing && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, h->stream);
    }
    ~PhaseScope()
    {
        if (h->timing && a && b) {
            cudaEventRecord(b, h->stream);
            h->recs.push_back({phase, a, b});
        }
    }
};

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return OTM_ERR_CUDA; \
    } while (0)

static size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// Carve every array out of the workspace. With base == NULL only the size is computed.
// Node arrays have nn_cap rows (room for inserted nodes); nn is the current count.
static size_t layout(int64_t nn, int64_t nn_cap, int64_t nm, int S, int precision, char *base, Dev *D,
                     int32_t **scan_tmp)
{
    size_t off = 0;
    const int64_t slots = nm * (int64_t)S;
    const int max_cells = (int)(16 * nn_cap + 65536);
#define TAKE(ptr, T, count)                                         \
    do {                                                            \
        if (base) (ptr) = (T *)(base + off);                        \
        off += a256((size_t)(count) * sizeof(T));                   \
    } while (0)
    Dev d;
    memset(&d, 0, sizeof(d));
    int32_t *tmp = nullptr;
    TAKE(d.err, unsigned long long, 1);
    TAKE(d.emax, int, 2);
    TAKE(d.grid, GridDev, 1);
    // nodes
    TAKE(d.x, double4_32a, nn_cap);
    TAKE(d.x_prev, double4_32a, nn_cap);
    TAKE(d.du, double4_32a, nn_cap);
    TAKE(d.mr, double4_32a, nn_cap);
    TAKE(d.spos, double4_32a, nn_cap);
    TAKE(d.spos32, float4, nn_cap);
    TAKE(d.du32, float4, nn_cap);
    TAKE(d.nflags, uint8_t, nn_cap);
    TAKE(d.ngid, int64_t, nn_cap);
    TAKE(d.ncount, int32_t, nn_cap);
    TAKE(d.noff, int32_t, nn_cap + 1);
    TAKE(d.node_cell, int32_t, nn_cap);
    TAKE(d.node_rank, int32_t, nn_cap);
    TAKE(d.sorted, int32_t, nn_cap);
    TAKE(d.cell_count, int32_t, (int64_t)max_cells + 1);
    TAKE(d.cell_start, int32_t, (int64_t)max_cells + 1);
    TAKE(tmp, int32_t, scan_tmp_ints((nn_cap > nm ? nn_cap : nm) + 1));
    // material points
    TAKE(d.xp, double4_32a, nm);
    TAKE(d.xp_prev, double4_32a, nm);
    TAKE(d.F, double, 9 * nm);
    TAKE(d.dF, double, 9 * nm);
    TAKE(d.be, double, 6 * nm);
    TAKE(d.sig, double, 6 * nm);
    TAKE(d.vol, double, nm);
    TAKE(d.mass, double, nm);
    TAKE(d.ebar, double, nm);
    TAKE(d.T, double, nm);
    TAKE(d.rate, double, nm);
    TAKE(d.lam, double, 3 * nm);
    TAKE(d.lam_prev, double, 3 * nm);
    TAKE(d.lam_prev2, double, 3 * nm);
    TAKE(d.lam_prev3, double, 3 * nm);
    TAKE(d.logz, double, nm);
    TAKE(d.logz_in, double, nm);
    TAKE(d.mat_id, int32_t, nm);
    TAKE(d.cnt, int32_t, nm);
    TAKE(d.newton_it, int32_t, nm);
    TAKE(d.failed, uint8_t, nm);
    TAKE(d.lme_fail, uint8_t, nm);
    TAKE(d.n_fail, int32_t, 1);
    TAKE(d.mgid, int64_t, nm);
    // pairs
    TAKE(d.ids, int32_t, slots);
    TAKE(d.shape, double4_32a, slots);
    if (precision == OTM_PRECISION_MIXED) {
        TAKE(d.contrib32, float4, slots);
    } else {
        TAKE(d.contrib64, double4_32a, slots);
    }
    TAKE(d.rank, uint16_t, slots);
    // staging of state transfers: up to 32 MiB, at least one 72-byte row
    size_t stage = (size_t)24 * (size_t)(nn_cap > nm ? nn_cap : nm);
    if (stage > ((size_t)32 << 20)) stage = (size_t)32 << 20;
    if (stage < 256) stage = 256;
    TAKE(d.stage, char, stage);
#undef TAKE
    if (base) {
        d.nn = nn;
        d.nm = nm;
        d.S = S;
        d.precision = precision;
        d.max_cells = max_cells;
        d.stage_bytes = stage;
        *D = d;
        *scan_tmp = tmp;
    }
    return off;
}

static int check_params(int64_t nn, int64_t nm, const otm_params *P)
{
    if (!P || nn <= 0 || nm <= 0) return OTM_ERR_ARG;
    if (P->max_support < 32 || P->max_support > kMaxS || (P->max_support % 32) != 0) return OTM_ERR_ARG;
    if (P->n_materials < 1 || P->n_materials > 4) return OTM_ERR_ARG;
    if (P->precision != OTM_PRECISION_FP64 && P->precision != OTM_PRECISION_MIXED) return OTM_ERR_ARG;
    if (!(P->h > 0) || !(P->beta > 0) || !(P->rs2 > 0) || !(P->dt > 0)) return OTM_ERR_ARG;
    if (!(P->cell_size * 2.0 >= sqrt(P->rs2))) return OTM_ERR_ARG;   // stencil of +-2 cells
    if (nm * (int64_t)P->max_support >= (int64_t)0x7fffffff) return OTM_ERR_ARG;
    if (nn >= (int64_t)0x7fffffff / 16) return OTM_ERR_ARG;
    if (!(P->eps_stab >= 0.0)) return OTM_ERR_ARG;
    if (P->max_insert < 0 || nn + P->max_insert >= (int64_t)0x7fffffff / 16) return OTM_ERR_ARG;
    return OTM_OK;
}

extern "C" int otm_workspace_bytes(int64_t n_nodes, int64_t n_mps, const otm_params *params, size_t *bytes)
{
    int st = check_params(n_nodes, n_mps, params);
    if (st != OTM_OK) return st;
    if (!bytes) return OTM_ERR_ARG;
    *bytes = layout(n_nodes, n_nodes + params->max_insert, n_mps, params->max_support, params->precision, nullptr,
                    nullptr, nullptr) + 256;
    return OTM_OK;
}

static void fill_params(Dev &D, const otm_params *P)
{
    D.h = P->h;
    D.beta = P->beta;
    D.rs2 = P->rs2;
    D.cell = P->cell_size;
    D.sc = make_search_const(P->cell_size, P->rs2);
    D.dt = P->dt;
    D.tol_abs = P->newton_tol * P->h;
    D.eps_stab = P->eps_stab;
    D.max_newton = P->max_newton;
    D.wall = P->wall;
    D.tool = P->tool;
    D.allow_erode = P->allow_erode;
    for (int i = 0; i < 3; i++) {
        D.wall_p[i] = P->wall_p[i];
        D.wall_n[i] = P->wall_n[i];
    }
    D.tool_x0 = P->tool_x0;
    D.tool_tip_y = P->tool_tip_y;
    D.tool_rake = P->tool_rake;
    D.tool_clear = P->tool_clear;
    D.tool_v = P->tool_v;
    D.friction = P->friction;
    for (int i = 0; i < 4; i++) D.mat[i] = P->mat[i];
}

static int read_error(otm_handle *h, int32_t *code, int64_t *id)
{
    unsigned long long key = 0;
    CK(cudaMemcpyAsync(&key, h->D.err, sizeof(key), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (key == ~0ULL) {
        if (code) *code = OTM_OK;
        if (id) *id = -1;
        return OTM_OK;
    }
    const int c = -(int)(key & 0xff);
    if (code) *code = c;
    if (id) *id = (int64_t)(key >> 8);
    return c;
}

// steps 5-6 of Algorithm 1 plus the node-major lists for the next step's step 1; with `insert`,
// MPs whose LME solve fails are flagged for node insertion instead of stopping the step
static int rebuild_supports(otm_handle *h, bool insert, int lme_mode)
{
    Dev &D = h->D;
    cudaStream_t s = h->stream;
    D.insert_mode = insert ? 1 : 0;
    D.lme_mode = lme_mode;
    {
        PhaseScope ps(h, OTM_PHASE_GRID);
        CK(launch_grid_build(D, s, &h->launches));
    }
    CK(cudaMemsetAsync(D.ncount, 0, (size_t)D.nn * sizeof(int32_t), s));
    CK(cudaMemsetAsync(D.emax, 0x80, 2 * sizeof(int), s));
    {
        PhaseScope ps(h, OTM_PHASE_SEARCH);
        CK(launch_search(D, s, &h->launches));
    }
    {
        PhaseScope ps(h, OTM_PHASE_NODE_MAJOR);
        CK(launch_node_offsets(D, h->scan_tmp, s, &h->launches));
    }
    {
        PhaseScope ps(h, OTM_PHASE_LME);
        CK(launch_lme(D, s, &h->launches));
    }
    D.insert_mode = 0;
    return OTM_OK;
}

// Node insertion after the LME solve of a step (rule in include/otm.h, otm_step): one node per
// flagged MP, then the search and solve once more for every MP, failures now being errors.
static int resolve_insertions(otm_handle *h)
{
    Dev &D = h->D;
    cudaStream_t s = h->stream;
    int32_t nf = 0;
    CK(cudaMemcpyAsync(&nf, D.n_fail, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nf == 0) return OTM_OK;
    {
        PhaseScope ps(h, OTM_PHASE_COMPACT);
        if (h->n_inserted + nf > h->P.max_insert) {
            CK(raise_flagged(D, OTM_ERR_CAPACITY, s, &h->launches));
        } else {
            CK(insert_nodes(D, h->scan_tmp, nf, h->nn0 + h->n_inserted, s, &h->launches));
            h->n_inserted += nf;
        }
        CK(cudaMemsetAsync(D.lme_fail, 0, (size_t)D.nm, s));
        CK(cudaMemsetAsync(D.n_fail, 0, sizeof(int32_t), s));
    }
    return rebuild_supports(h, false, kLmeKeep);
}

extern "C" int otm_init(const otm_problem *prob, const otm_params *params, void *stream, void *workspace,
                        size_t ws_bytes, otm_handle **out)
{
    if (!prob || !params || !out || !workspace) return OTM_ERR_ARG;
    *out = nullptr;
    const int64_t nn = prob->n_nodes, nm = prob->n_mps;
    int st = check_params(nn, nm, params);
    if (st != OTM_OK) return st;
    if (!prob->node_x || !prob->node_du0 || !prob->node_flags || !prob->mp_x || !prob->mp_vol || !prob->mp_mass ||
        !prob->mp_material)
        return OTM_ERR_ARG;
    for (int64_t p = 0; p < nm; p++)
        if (prob->mp_material[p] < 0 || prob->mp_material[p] >= params->n_materials) return OTM_ERR_ARG;
    if (((uintptr_t)workspace) & 255) return OTM_ERR_ARG;
    if (exp_table_setup() != cudaSuccess) return OTM_ERR_CUDA;
    const int64_t nn_cap = nn + params->max_insert;
    size_t need = layout(nn, nn_cap, nm, params->max_support, params->precision, nullptr, nullptr, nullptr);
    if (ws_bytes < need) return OTM_ERR_WORKSPACE;

    otm_handle *h = new (std::nothrow) otm_handle();
    if (!h) return OTM_ERR_ARG;
    h->P = *params;
    h->stream = (cudaStream_t)stream;
    h->ws = workspace;
    h->ws_bytes = ws_bytes;
    layout(nn, nn_cap, nm, params->max_support, params->precision, (char *)workspace, &h->D, &h->scan_tmp);
    fill_params(h->D, params);
    h->nn0 = nn;
    h->nm0 = nm;
    h->nn_cap = nn_cap;
    Dev &D = h->D;
    cudaStream_t s = h->stream;
    int rc = OTM_OK;
    do {
        // host problem -> workspace (positions staged through the pair-shape region)
        double *stage = (double *)D.shape;
        if ((size_t)nm * D.S * sizeof(double4_32a) < (size_t)3 * (nn > nm ? nn : nm) * sizeof(double)) {
            rc = OTM_ERR_ARG;
            break;
        }
        if (cudaMemsetAsync(D.err, 0xff, sizeof(unsigned long long), s) != cudaSuccess ||
            cudaMemsetAsync(D.lme_fail, 0, (size_t)nm, s) != cudaSuccess ||
            cudaMemsetAsync(D.n_fail, 0, sizeof(int32_t), s) != cudaSuccess) {
            rc = OTM_ERR_CUDA;
            break;
        }
        if (cudaMemcpyAsync(stage, prob->node_x, 24 * nn, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            launch_pack3to4(stage, nn, D.x, s, &h->launches) != cudaSuccess ||
            cudaMemcpyAsync(stage, prob->node_du0, 24 * nn, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            launch_pack3to4(stage, nn, D.du, s, &h->launches) != cudaSuccess ||
            cudaMemcpyAsync(stage, prob->mp_x, 24 * nm, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            launch_pack3to4(stage, nm, D.xp, s, &h->launches) != cudaSuccess ||
            cudaMemcpyAsync(D.nflags, prob->node_flags, nn, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(D.vol, prob->mp_vol, 8 * nm, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(D.mass, prob->mp_mass, 8 * nm, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(D.mat_id, prob->mp_material, 4 * nm, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            launch_init_state(D, params->T0, s, &h->launches) != cudaSuccess) {
            rc = OTM_ERR_CUDA;
            break;
        }
        // the staging copies must land before the region is reused by the support build
        if (cudaStreamSynchronize(s) != cudaSuccess) { rc = OTM_ERR_CUDA; break; }
        rc = rebuild_supports(h, false, kLmePlain);
        if (rc != OTM_OK) break;
        rc = read_error(h, nullptr, nullptr);
    } while (0);
    if (rc != OTM_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return OTM_OK;
}

static int enqueue_step(otm_handle *h)
{
    Dev &D = h->D;
    cudaStream_t s = h->stream;
    const double t_next = (double)(h->step + 1) * D.dt;
    {   // 1-2: lumped mass / force (segmented reduction), central difference, contact, x update
        PhaseScope ps(h, OTM_PHASE_NODE_UPDATE);
        CK(launch_node_update(D, t_next, s, &h->launches));
    }
    if (h->frozen) {
        // frozen topology: kinematics (3) and return map (4) over the supports the step starts
        // with, then the LME (6) at the new positions over the same supports and lists
        {
            PhaseScope ps(h, OTM_PHASE_KINEMATICS);
            CK(launch_kinematics(D, s, &h->launches));
        }
        {
            PhaseScope ps(h, OTM_PHASE_RETURN_MAP);
            CK(launch_return_map(D, s, &h->launches));
        }
        CK(cudaMemsetAsync(D.emax, 0x80, 2 * sizeof(int), s));
        {
            PhaseScope ps(h, OTM_PHASE_LME);
            D.lme_mode = kLmeStep;
            CK(launch_lme(D, s, &h->launches));
        }
        h->step++;
        return OTM_OK;
    }
    if (!D.allow_erode) {
        // no MP can leave the body within the step: the kinematics gather (3) and the search at
        // the new MP position (5) run in one kernel, then the return map (4) and the LME (6)
        {
            PhaseScope ps(h, OTM_PHASE_GRID);
            CK(launch_grid_build(D, s, &h->launches));
        }
        CK(cudaMemsetAsync(D.ncount, 0, (size_t)D.nn * sizeof(int32_t), s));
        CK(cudaMemsetAsync(D.emax, 0x80, 2 * sizeof(int), s));
        {
            PhaseScope ps(h, OTM_PHASE_SEARCH);
            CK(launch_kin_search(D, s, &h->launches));
        }
        {
            PhaseScope ps(h, OTM_PHASE_NODE_MAJOR);
            CK(launch_node_offsets(D, h->scan_tmp, s, &h->launches));
        }
        {
            PhaseScope ps(h, OTM_PHASE_RETURN_MAP);
            CK(launch_return_map(D, s, &h->launches));
        }
        {
            PhaseScope ps(h, OTM_PHASE_LME);
            D.insert_mode = h->P.max_insert > 0 ? 1 : 0;
            D.lme_mode = kLmeStep;
            CK(launch_lme(D, s, &h->launches));
            D.insert_mode = 0;
        }
        if (h->P.max_insert > 0) {
            int rc = resolve_insertions(h);
            if (rc != OTM_OK) return rc;
        }
        h->step++;
        return OTM_OK;
    }
    {   // 3: MP position, F increment
        PhaseScope ps(h, OTM_PHASE_KINEMATICS);
        CK(launch_kinematics(D, s, &h->launches));
    }
    {   // 4: constitutive update
        PhaseScope ps(h, OTM_PHASE_RETURN_MAP);
        CK(launch_return_map(D, s, &h->launches));
    }
    int64_t eroded = 0;
    {   // fracture: failed MPs leave before the new supports are built
        PhaseScope ps(h, OTM_PHASE_COMPACT);
        CK(erode_mps(D, h->scan_tmp, &eroded, s, &h->launches));
        h->n_eroded += eroded;
    }
    // 5-6: linked-cell search, LME shape functions, contributions, node-major lists
    int rc = rebuild_supports(h, h->P.max_insert > 0, kLmeStep);
    if (rc != OTM_OK) return rc;
    if (h->P.max_insert > 0 && (rc = resolve_insertions(h)) != OTM_OK) return rc;
    if (eroded > 0) {      // nodes left in no support are removed
        PhaseScope ps(h, OTM_PHASE_COMPACT);
        int64_t removed = 0;
        CK(remove_orphan_nodes(D, h->scan_tmp, &removed, s, &h->launches));
        h->n_removed += removed;
    }
    h->step++;
    return OTM_OK;
}

extern "C" int otm_step_async(otm_handle *h, int32_t n_steps)
{
    if (!h || n_steps < 0) return OTM_ERR_ARG;
    for (int32_t k = 0; k < n_steps; k++) {
        int rc = enqueue_step(h);
        if (rc != OTM_OK) return rc;
    }
    return OTM_OK;
}

extern "C" int otm_step(otm_handle *h, int32_t n_steps)
{
    int rc = otm_step_async(h, n_steps);
    if (rc != OTM_OK) return rc;
    return read_error(h, nullptr, nullptr);
}

extern "C" int otm_error_detail(otm_handle *h, int32_t *code, int64_t *first_id)
{
    if (!h) return OTM_ERR_ARG;
    int c = 0;
    int64_t id = -1;
    int rc = read_error(h, &c, &id);
    if (rc == OTM_ERR_CUDA) return rc;
    if (code) *code = c;
    if (first_id) *first_id = id;
    return OTM_OK;
}

extern "C" int otm_counts(otm_handle *h, int64_t *n_nodes, int64_t *n_mps, int64_t *n_pairs, int64_t *step)
{
    if (!h) return OTM_ERR_ARG;
    if (n_nodes) *n_nodes = h->D.nn;
    if (n_mps) *n_mps = h->D.nm;
    if (step) *step = h->step;
    if (n_pairs) {
        int32_t tot = 0;
        CK(cudaMemcpyAsync(&tot, h->D.noff + h->D.nn, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        *n_pairs = tot;
    }
    return OTM_OK;
}

extern "C" int otm_kernel_launches(otm_handle *h, int64_t *launches)
{
    if (!h || !launches) return OTM_ERR_ARG;
    *launches = h->launches;
    return OTM_OK;
}

struct FieldView {
    const void *src;   // device base
    size_t pitch;      // device row pitch
    size_t width;      // bytes per row copied
    size_t rows;
};

static bool field_view(otm_handle *h, int32_t f, FieldView *v)
{
    const Dev &D = h->D;
    const size_t nn = (size_t)D.nn, nm = (size_t)D.nm, S = (size_t)D.S;
    switch (f) {
    case OTM_FIELD_NODE_X: *v = {D.x, 32, 24, nn}; return true;
    case OTM_FIELD_NODE_DU: *v = {D.du, 32, 24, nn}; return true;
    case OTM_FIELD_NODE_MASS: *v = {D.mr, 32, 8, nn}; return true;
    case OTM_FIELD_NODE_FORCE: *v = {(const char *)D.mr + 8, 32, 24, nn}; return true;
    case OTM_FIELD_NODE_FLAGS: *v = {D.nflags, 1, 1, nn}; return true;
    case OTM_FIELD_MP_X: *v = {D.xp, 32, 24, nm}; return true;
    case OTM_FIELD_F: *v = {D.F, 72, 72, nm}; return true;
    case OTM_FIELD_DF: *v = {D.dF, 72, 72, nm}; return true;
    case OTM_FIELD_BE: *v = {D.be, 48, 48, nm}; return true;
    case OTM_FIELD_SIGMA: *v = {D.sig, 48, 48, nm}; return true;
    case OTM_FIELD_VOL: *v = {D.vol, 8, 8, nm}; return true;
    case OTM_FIELD_EBAR: *v = {D.ebar, 8, 8, nm}; return true;
    case OTM_FIELD_T: *v = {D.T, 8, 8, nm}; return true;
    case OTM_FIELD_RATE: *v = {D.rate, 8, 8, nm}; return true;
    case OTM_FIELD_LAMBDA: *v = {D.lam, 24, 24, nm}; return true;
    case OTM_FIELD_SUPPORT_COUNT: *v = {D.cnt, 4, 4, nm}; return true;
    case OTM_FIELD_NEWTON_IT: *v = {D.newton_it, 4, 4, nm}; return true;
    case OTM_FIELD_SUPPORT_IDS: *v = {D.ids, 4 * S, 4 * S, nm}; return true;
    case OTM_FIELD_SHAPE: *v = {D.shape, 32 * S, 32 * S, nm}; return true;
    case OTM_FIELD_MP_GID: *v = {D.mgid, 8, 8, nm}; return true;
    case OTM_FIELD_NODE_GID: *v = {D.ngid, 8, 8, nn}; return true;
    default: return false;
    }
}

// device rows (pitch) <-> dense host rows (width), through the staging buffer in chunks
static int rows_d2h(otm_handle *h, const void *src, size_t pitch, size_t width, size_t rows, void *host_dst)
{
    const size_t chunk = h->D.stage_bytes / width;
    for (size_t r0 = 0; r0 < rows; r0 += chunk) {
        const size_t n = (rows - r0 < chunk) ? rows - r0 : chunk;
        CK(launch_rows_to_dense((const char *)src + r0 * pitch, pitch, width, (int64_t)n, h->D.stage, h->stream));
        CK(cudaMemcpyAsync((char *)host_dst + r0 * width, h->D.stage, n * width, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return OTM_OK;
}

static int rows_h2d(otm_handle *h, const void *host_src, size_t pitch, size_t width, size_t rows, void *dst)
{
    const size_t chunk = h->D.stage_bytes / width;
    for (size_t r0 = 0; r0 < rows; r0 += chunk) {
        const size_t n = (rows - r0 < chunk) ? rows - r0 : chunk;
        CK(cudaMemcpyAsync(h->D.stage, (const char *)host_src + r0 * width, n * width, cudaMemcpyHostToDevice,
                           h->stream));
        CK(launch_rows_from_dense(h->D.stage, pitch, width, (int64_t)n, (char *)dst + r0 * pitch, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return OTM_OK;
}

extern "C" int otm_state(otm_handle *h, int32_t field, void *host_dst, size_t bytes)
{
    if (!h || !host_dst) return OTM_ERR_ARG;
    FieldView v;
    if (!field_view(h, field, &v)) return OTM_ERR_ARG;
    if (bytes != v.width * v.rows) return OTM_ERR_ARG;
    if (v.rows == 0) return OTM_OK;
    if (v.pitch == v.width) {
        CK(cudaMemcpyAsync(host_dst, v.src, bytes, cudaMemcpyDeviceToHost, h->stream));
    } else {   // pitched rows: packed on the device in chunks, each chunk one contiguous copy
        const int rc = rows_d2h(h, v.src, v.pitch, v.width, v.rows, host_dst);
        if (rc != OTM_OK) return rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    if (field == OTM_FIELD_SUPPORT_IDS || field == OTM_FIELD_SHAPE) {
        // rows are stored in linked-cell order; the export orders each row by node ID
        const size_t nm = (size_t)h->D.nm, S = (size_t)h->D.S;
        std::vector<int32_t> cnt(nm), ids;
        CK(cudaMemcpy(cnt.data(), h->D.cnt, nm * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (field == OTM_FIELD_SUPPORT_IDS) {
            int32_t *row = (int32_t *)host_dst;
            for (size_t p = 0; p < nm; p++) std::sort(row + p * S, row + p * S + cnt[p]);
        } else {
            ids.resize(nm * S);
            CK(cudaMemcpy(ids.data(), h->D.ids, nm * S * sizeof(int32_t), cudaMemcpyDeviceToHost));
            double *sh = (double *)host_dst;
            std::vector<int> perm;
            std::vector<double> tmp;
            for (size_t p = 0; p < nm; p++) {
                const int n = cnt[p];
                perm.resize(n);
                std::iota(perm.begin(), perm.end(), 0);
                const int32_t *r = ids.data() + p * S;
                std::sort(perm.begin(), perm.end(), [r](int a, int b) { return r[a] < r[b]; });
                tmp.assign(sh + 4 * p * S, sh + 4 * (p * S + n));
                for (int k = 0; k < n; k++)
                    for (int c = 0; c < 4; c++) sh[4 * (p * S + k) + c] = tmp[4 * perm[k] + c];
            }
        }
    }
    return OTM_OK;
}

extern "C" int otm_state_rows(otm_handle *h, int32_t field, const int64_t *rows, int64_t n_rows, void *host_dst,
                              size_t bytes)
{
    if (!h || !rows || !host_dst || n_rows < 0) return OTM_ERR_ARG;
    FieldView v;
    if (!field_view(h, field, &v)) return OTM_ERR_ARG;
    if (bytes != v.width * (size_t)n_rows) return OTM_ERR_ARG;
    for (int64_t r = 0; r < n_rows; r++) {
        if (rows[r] < 0 || (size_t)rows[r] >= v.rows) return OTM_ERR_ARG;
        CK(cudaMemcpyAsync((char *)host_dst + (size_t)r * v.width, (const char *)v.src + (size_t)rows[r] * v.pitch,
                           v.width, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    if (field == OTM_FIELD_SUPPORT_IDS || field == OTM_FIELD_SHAPE) {   // order each row by node ID
        const size_t S = (size_t)h->D.S;
        std::vector<int32_t> cnt(n_rows), ids(S);
        for (int64_t r = 0; r < n_rows; r++) {
            CK(cudaMemcpy(&cnt[r], h->D.cnt + rows[r], sizeof(int32_t), cudaMemcpyDeviceToHost));
            const int n = cnt[r];
            if (field == OTM_FIELD_SUPPORT_IDS) {
                int32_t *row = (int32_t *)host_dst + (size_t)r * S;
                std::sort(row, row + n);
            } else {
                CK(cudaMemcpy(ids.data(), h->D.ids + (size_t)rows[r] * S, S * sizeof(int32_t), cudaMemcpyDeviceToHost));
                std::vector<int> perm(n);
                std::iota(perm.begin(), perm.end(), 0);
                std::sort(perm.begin(), perm.end(), [&](int a, int b) { return ids[a] < ids[b]; });
                double *sh = (double *)host_dst + (size_t)r * S * 4;
                std::vector<double> tmp(sh, sh + 4 * (size_t)n);
                for (int k = 0; k < n; k++)
                    for (int c = 0; c < 4; c++) sh[4 * k + c] = tmp[4 * perm[k] + c];
            }
        }
    }
    return OTM_OK;
}

extern "C" int otm_set_state(otm_handle *h, int32_t field, const void *host_src, size_t bytes)
{
    if (!h || !host_src) return OTM_ERR_ARG;
    switch (field) {
    case OTM_FIELD_NODE_X: case OTM_FIELD_NODE_DU: case OTM_FIELD_MP_X: case OTM_FIELD_F:
    case OTM_FIELD_BE: case OTM_FIELD_SIGMA: case OTM_FIELD_VOL: case OTM_FIELD_EBAR: case OTM_FIELD_T:
    case OTM_FIELD_LAMBDA: break;
    default: return OTM_ERR_ARG;
    }
    FieldView v;
    field_view(h, field, &v);
    if (bytes != v.width * v.rows) return OTM_ERR_ARG;
    if (v.pitch == v.width) {
        CK(cudaMemcpyAsync((void *)v.src, host_src, bytes, cudaMemcpyHostToDevice, h->stream));
    } else {
        const int rc = rows_h2d(h, host_src, v.pitch, v.width, v.rows, (void *)v.src);
        if (rc != OTM_OK) return rc;
    }
    if (field == OTM_FIELD_NODE_DU)   // keep the FP32 copy of the increments in step
        CK(launch_du_to_f32(h->D, h->stream, &h->launches));
    CK(cudaStreamSynchronize(h->stream));
    return OTM_OK;
}

extern "C" int otm_refresh(otm_handle *h)
{
    if (!h) return OTM_ERR_ARG;
    CK(cudaMemsetAsync(h->D.err, 0xff, sizeof(unsigned long long), h->stream));
    int rc = rebuild_supports(h, false, kLmePlain);
    if (rc != OTM_OK) return rc;
    return read_error(h, nullptr, nullptr);
}

extern "C" int otm_freeze_topology(otm_handle *h, int32_t on)
{
    if (!h) return OTM_ERR_ARG;
    if (on && (h->P.allow_erode || h->P.max_insert > 0)) return OTM_ERR_ARG;
    h->frozen = on != 0;
    return OTM_OK;
}

extern "C" int otm_step_with_supports(otm_handle *h, const int32_t *counts, const int32_t *ids)
{
    if (!h || !counts || !ids) return OTM_ERR_ARG;
    if (h->P.allow_erode || h->P.max_insert > 0) return OTM_ERR_ARG;
    Dev &D = h->D;
    const int64_t nm = D.nm, S = D.S, nn = D.nn;
    for (int64_t p = 0; p < nm; p++) {
        if (counts[p] < 1 || counts[p] > S) return OTM_ERR_ARG;
        const int32_t *row = ids + p * S;
        for (int32_t k = 0; k < counts[p]; k++)
            if (row[k] < 0 || row[k] >= nn) return OTM_ERR_ARG;
    }
    cudaStream_t s = h->stream;
    const double t_next = (double)(h->step + 1) * D.dt;
    {
        PhaseScope ps(h, OTM_PHASE_NODE_UPDATE);
        CK(launch_node_update(D, t_next, s, &h->launches));
    }
    {   // kinematics over the supports of the state the step starts from
        PhaseScope ps(h, OTM_PHASE_KINEMATICS);
        CK(launch_kinematics(D, s, &h->launches));
    }
    {
        PhaseScope ps(h, OTM_PHASE_RETURN_MAP);
        CK(launch_return_map(D, s, &h->launches));
    }
    // the given supports of the new state (stream-ordered after the kinematics read the old ones)
    CK(cudaMemcpyAsync(D.cnt, counts, (size_t)nm * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(D.ids, ids, (size_t)(nm * S) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(D.ncount, 0, (size_t)nn * sizeof(int32_t), s));
    CK(cudaMemsetAsync(D.emax, 0x80, 2 * sizeof(int), s));
    CK(launch_rebuild_ranks(D, s, &h->launches));
    {
        PhaseScope ps(h, OTM_PHASE_NODE_MAJOR);
        CK(launch_node_offsets(D, h->scan_tmp, s, &h->launches));
    }
    {
        PhaseScope ps(h, OTM_PHASE_LME);
        D.lme_mode = kLmeStep;
        CK(launch_lme(D, s, &h->launches));
    }
    h->step++;
    return read_error(h, nullptr, nullptr);
}

extern "C" int otm_phase_timing(otm_handle *h, int32_t enable)
{
    if (!h) return OTM_ERR_ARG;
    h->timing = enable != 0;
    return OTM_OK;
}

extern "C" int otm_phase_times(otm_handle *h, double *ms, int64_t *launches)
{
    if (!h) return OTM_ERR_ARG;
    CK(cudaStreamSynchronize(h->stream));
    for (auto &r : h->recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            h->phase_ms[r.phase] += t;
            h->phase_n[r.phase] += 1;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    h->recs.clear();
    for (int i = 0; i < OTM_N_PHASES; i++) {
        if (ms) ms[i] = h->phase_ms[i];
        if (launches) launches[i] = h->phase_n[i];
        h->phase_ms[i] = 0.0;
        h->phase_n[i] = 0;
    }
    return OTM_OK;
}

extern "C" void otm_destroy(otm_handle *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto &r : h->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete h;
}

// ------------------------------------------------------------------ snapshots
// A snapshot holds everything a step reads except what the LME kernel regenerates bit for bit
// (shape functions, node-major contributions, ranks, offsets): node and MP state, the support
// lists, and the exponent shift the last LME solve used.
struct SnapHeader {
    int64_t nn, nm, step, magic, n_inserted;
    int64_t nn_cap, nm_cap, S;     // the layout the snapshot was written with
};
struct SnapField {
    void *p;
    size_t row;
    int kind;   // 0 node rows, 1 MP rows, 2 padded pair rows
};

static int snap_fields(otm_handle *h, SnapField *f)
{
    Dev &D = h->D;
    const size_t S = (size_t)D.S;
    int k = 0;
    f[k++] = {D.x, 32, 0}; f[k++] = {D.x_prev, 32, 0}; f[k++] = {D.du, 32, 0}; f[k++] = {D.du32, 16, 0};
    f[k++] = {D.nflags, 1, 0}; f[k++] = {D.ngid, 8, 0};
    f[k++] = {D.xp, 32, 1}; f[k++] = {D.xp_prev, 32, 1}; f[k++] = {D.F, 72, 1}; f[k++] = {D.dF, 72, 1}; f[k++] = {D.be, 48, 1};
    f[k++] = {D.sig, 48, 1}; f[k++] = {D.vol, 8, 1}; f[k++] = {D.mass, 8, 1}; f[k++] = {D.ebar, 8, 1};
    f[k++] = {D.T, 8, 1}; f[k++] = {D.rate, 8, 1}; f[k++] = {D.lam, 24, 1}; f[k++] = {D.lam_prev, 24, 1}; f[k++] = {D.lam_prev2, 24, 1}; f[k++] = {D.lam_prev3, 24, 1};
    f[k++] = {D.logz, 8, 1};
    f[k++] = {D.logz_in, 8, 1}; f[k++] = {D.mat_id, 4, 1}; f[k++] = {D.mgid, 8, 1}; f[k++] = {D.cnt, 4, 1};
    f[k++] = {D.newton_it, 4, 1}; f[k++] = {D.failed, 1, 1};
    f[k++] = {D.ids, 4 * S, 1};
    return k;
}

static size_t snap_size(otm_handle *h)
{
    SnapField f[32];
    const int n = snap_fields(h, f);
    size_t b = 256;
    for (int i = 0; i < n; i++) b += a256(f[i].row * (size_t)(f[i].kind == 0 ? h->nn_cap : h->nm0));
    return b;
}

extern "C" int otm_snapshot_bytes(otm_handle *h, size_t *bytes)
{
    if (!h || !bytes) return OTM_ERR_ARG;
    *bytes = snap_size(h);
    return OTM_OK;
}

extern "C" int otm_snapshot_save(otm_handle *h, void *dst)
{
    if (!h || !dst || (((uintptr_t)dst) & 255)) return OTM_ERR_ARG;
    SnapField f[32];
    const int n = snap_fields(h, f);
    SnapHeader hd = {h->D.nn, h->D.nm, h->step, 0x4f544d53, h->n_inserted, h->nn_cap, h->nm0, h->D.S};
    CK(cudaMemcpyAsync(dst, &hd, sizeof(hd), cudaMemcpyDefault, h->stream));
    char *o = (char *)dst + 256;
    for (int i = 0; i < n; i++) {
        const size_t rows = (size_t)(f[i].kind == 0 ? h->D.nn : h->D.nm);
        CK(cudaMemcpyAsync(o, f[i].p, f[i].row * rows, cudaMemcpyDefault, h->stream));
        o += a256(f[i].row * (size_t)(f[i].kind == 0 ? h->nn_cap : h->nm0));
    }
    CK(cudaStreamSynchronize(h->stream));
    return OTM_OK;
}

extern "C" int otm_snapshot_load(otm_handle *h, const void *src)
{
    if (!h || !src || (((uintptr_t)src) & 255)) return OTM_ERR_ARG;
    SnapHeader hd;
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(&hd, src, sizeof(hd), cudaMemcpyDefault));
    if (hd.magic != 0x4f544d53 || hd.nn > h->nn_cap || hd.nm > h->nm0) return OTM_ERR_ARG;
    if (hd.nn_cap != h->nn_cap || hd.nm_cap != h->nm0 || hd.S != h->D.S) return OTM_ERR_ARG;
    h->D.nn = hd.nn;
    h->D.nm = hd.nm;
    h->step = hd.step;
    h->n_inserted = hd.n_inserted;
    SnapField f[32];
    const int n = snap_fields(h, f);
    const char *o = (const char *)src + 256;
    for (int i = 0; i < n; i++) {
        const size_t rows = (size_t)(f[i].kind == 0 ? h->D.nn : h->D.nm);
        CK(cudaMemcpyAsync(f[i].p, o, f[i].row * rows, cudaMemcpyDefault, h->stream));
        o += a256(f[i].row * (size_t)(f[i].kind == 0 ? h->nn_cap : h->nm0));
    }
    Dev &D = h->D;
    // the FP32 copy of the increments from the FP64 one (a snapshot of either precision path
    // loads into either)
    CK(launch_du_to_f32(D, h->stream, &h->launches));
    // regenerate ranks, offsets, shape functions and contributions: the LME restarts from the
    // stored lambda with the stored exponent shift, so it reproduces them exactly
    CK(cudaMemsetAsync(D.err, 0xff, sizeof(unsigned long long), h->stream));
    CK(cudaMemsetAsync(D.ncount, 0, (size_t)D.nn * sizeof(int32_t), h->stream));
    CK(cudaMemsetAsync(D.emax, 0x80, 2 * sizeof(int), h->stream));
    CK(launch_rebuild_ranks(D, h->stream, &h->launches));
    CK(launch_node_offsets(D, h->scan_tmp, h->stream, &h->launches));
    CK(cudaMemcpyAsync(D.logz, D.logz_in, (size_t)D.nm * 8, cudaMemcpyDeviceToDevice, h->stream));
    D.lme_mode = kLmeKeep;
    CK(launch_lme(D, h->stream, &h->launches));
    return read_error(h, nullptr, nullptr);
}

// ------------------------------------------------------------------ adjoint
static size_t adj_layout(otm_handle *h, char *base, AdjDev *A)
{
    const int64_t nn = h->nn0, nm = h->nm0, slots = nm * (int64_t)h->D.S;
    size_t off = 256;
#define ATAKE(ptr, T, count)                                        \
    do {                                                            \
        if (base) A->ptr = (T *)(base + off);                       \
        off += a256((size_t)(count) * sizeof(T));                   \
    } while (0)
    ATAKE(xb, double4_32a, nn); ATAKE(dub, double4_32a, nn); ATAKE(rb, double4_32a, nn);
    ATAKE(Fb, double, 9 * nm); ATAKE(beb, double, 6 * nm); ATAKE(ebb, double, nm); ATAKE(Tb, double, nm);
    ATAKE(vb, double, nm); ATAKE(sigb, double, 6 * nm); ATAKE(dFb, double, 9 * nm); ATAKE(thb, double, 5 * nm);
    ATAKE(xpb, double4_32a, nm);
    ATAKE(pb_cur, double4_32a, slots); ATAKE(pb_prev, double4_32a, slots);
    ATAKE(du_n, double4_32a, nn);
    ATAKE(F_n, double, 9 * nm); ATAKE(be_n, double, 6 * nm); ATAKE(ebar_n, double, nm); ATAKE(T_n, double, nm);
    ATAKE(vol_n, double, nm); ATAKE(sig_n, double, 6 * nm);
    ATAKE(shape_n, double4_32a, slots); ATAKE(ids_n, int32_t, slots); ATAKE(cnt_n, int32_t, nm);
    ATAKE(noff_n, int32_t, nn + 1); ATAKE(rank_n, uint16_t, slots);
    ATAKE(sc1, double4_32a, slots); ATAKE(sc3a, double4_32a, slots); ATAKE(sc3b, double4_32a, slots);
#undef ATAKE
    return off;
}

static AdjDev adj_view(otm_handle *h)
{
    AdjDev A;
    memset(&A, 0, sizeof(A));
    adj_layout(h, (char *)h->adj_ws, &A);
    if (h->adj_swap) {
        double4_32a *t = A.pb_cur;
        A.pb_cur = A.pb_prev;
        A.pb_prev = t;
    }
    return A;
}

extern "C" int otm_adjoint_bytes(otm_handle *h, size_t *bytes)
{
    if (!h || !bytes) return OTM_ERR_ARG;
    AdjDev A;
    *bytes = adj_layout(h, nullptr, &A);
    return OTM_OK;
}

extern "C" int otm_adjoint_begin(otm_handle *h, void *adj_ws, size_t bytes, const double *xbar_host)
{
    if (!h || !adj_ws || !xbar_host || (((uintptr_t)adj_ws) & 255)) return OTM_ERR_ARG;
    AdjDev A;
    const size_t need = adj_layout(h, nullptr, &A);
    if (bytes < need) return OTM_ERR_WORKSPACE;
    if (h->P.allow_erode || h->P.max_insert > 0) return OTM_ERR_ARG;   // the adjoint keeps the node and MP sets fixed
    if (h->P.eps_stab != 0.0) return OTM_ERR_ARG;   // the stabilisation term is not differentiated
    h->adj_ws = adj_ws;
    h->adj_swap = false;
    CK(cudaMemsetAsync(adj_ws, 0, need, h->stream));
    A = adj_view(h);
    const int rc = rows_h2d(h, xbar_host, 32, 24, (size_t)h->D.nn, A.xb);
    if (rc != OTM_OK) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return OTM_OK;
}

extern "C" int otm_adjoint_step(otm_handle *h, void *adj_ws, const void *next_snapshot)
{
    if (!h || !adj_ws || adj_ws != h->adj_ws) return OTM_ERR_ARG;
    AdjDev A = adj_view(h);
    Dev &D = h->D;
    cudaStream_t s = h->stream;
    const size_t nn = (size_t)D.nn, nm = (size_t)D.nm, slots = nm * (size_t)D.S;
    // copies of state n that the recomputed step overwrites
    CK(cudaMemcpyAsync(A.du_n, D.du, 32 * nn, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.F_n, D.F, 72 * nm, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.be_n, D.be, 48 * nm, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.ebar_n, D.ebar, 8 * nm, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.T_n, D.T, 8 * nm, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.vol_n, D.vol, 8 * nm, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.sig_n, D.sig, 48 * nm, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.shape_n, D.shape, 32 * slots, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.ids_n, D.ids, 4 * slots, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.cnt_n, D.cnt, 4 * nm, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.rank_n, D.rank, 2 * slots, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(A.noff_n, D.noff, 4 * (nn + 1), cudaMemcpyDeviceToDevice, s));
    if (next_snapshot) {
        // the node update of step n (its masses and forces feed the node adjoint), then state
        // n+1 from its snapshot (the update's positions and increments are the snapshot's)
        {
            PhaseScope ps(h, OTM_PHASE_NODE_UPDATE);
            CK(launch_node_update(D, (double)(h->step + 1) * D.dt, s, &h->launches));
        }
        const int rc = otm_snapshot_load(h, next_snapshot);
        if (rc != OTM_OK) return rc;
    } else {
        // step n again (deterministic: reproduces the trajectory)
        const int rc = enqueue_step(h);
        if (rc != OTM_OK) return rc;
    }
    CK(launch_adjoint_backward(D, A, s, &h->launches));
    h->adj_swap = !h->adj_swap;   // the adjoint of shape n becomes the current pair adjoint
    return read_error(h, nullptr, nullptr);
}

extern "C" int otm_adjoint_result(otm_handle *h, void *adj_ws, double *theta_bar, double *dubar_host)
{
    if (!h || !adj_ws || adj_ws != h->adj_ws || !theta_bar) return OTM_ERR_ARG;
    AdjDev A = adj_view(h);
    const size_t nm = (size_t)h->D.nm;
    std::vector<double> th(5 * nm);
    CK(cudaMemcpyAsync(th.data(), A.thb, 5 * nm * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (dubar_host) {
        const int rc = rows_d2h(h, A.dub, 32, 24, (size_t)h->D.nn, dubar_host);
        if (rc != OTM_OK) return rc;
    }
    for (int k = 0; k < 5; k++) theta_bar[k] = 0.0;
    for (size_t p = 0; p < nm; p++)   // fixed order: deterministic
        for (int k = 0; k < 5; k++) theta_bar[k] += th[5 * p + k];
    return OTM_OK;
}

// ------------------------------------------------------------------ stand-alone entries
extern "C" int otm_search_scratch_bytes(int64_t n_nodes, size_t *bytes)
{
    if (n_nodes <= 0 || !bytes) return OTM_ERR_ARG;
    *bytes = search_scratch_bytes(n_nodes);
    return OTM_OK;
}

extern "C" int otm_support_search(const double *node_x, int64_t n_nodes, const double *mp_x, int64_t n_mps,
                                  double rs2, double cell_size, int32_t max_support, int32_t *ids, int32_t *counts,
                                  void *scratch, size_t scratch_bytes, double *grid_out, int32_t *status,
                                  void *stream)
{
    if (!node_x || !mp_x || !ids || !counts || !scratch || !status || n_nodes <= 0 || n_mps < 0) return OTM_ERR_ARG;
    if (max_support < 1 || max_support > kMaxS) return OTM_ERR_ARG;
    if (!(rs2 > 0) || !(cell_size * 2.0 >= sqrt(rs2))) return OTM_ERR_ARG;
    if (((uintptr_t)scratch) & 255) return OTM_ERR_ARG;
    if (scratch_bytes < search_scratch_bytes(n_nodes)) return OTM_ERR_WORKSPACE;
    CK(launch_search_only(node_x, n_nodes, mp_x, n_mps, rs2, cell_size, max_support, ids, counts, scratch,
                          scratch_bytes, grid_out, status, (cudaStream_t)stream));
    return OTM_OK;
}

extern "C" int otm_lme(const double *node_x, const double *mp_x, int64_t n_mps, const int32_t *ids,
                       const int32_t *counts, int32_t max_support, double beta, double tol_abs, int32_t max_newton,
                       double *lambda, double *shape, int32_t *iters, int32_t *status, void *stream)
{
    if (!node_x || !mp_x || !ids || !counts || !lambda || !shape || !status || n_mps < 0) return OTM_ERR_ARG;
    if (max_support < 1 || max_support > kMaxS || !(beta > 0) || !(tol_abs > 0)) return OTM_ERR_ARG;
    CK(exp_table_setup());
    CK(launch_lme_only(node_x, mp_x, n_mps, ids, counts, max_support, beta, tol_abs, max_newton, lambda, shape,
                       iters, status, (cudaStream_t)stream));
    return OTM_OK;
}

extern "C" int otm_exp_selftest(const double *x, int64_t n, double *mine, double *ref, void *stream)
{
    if (!x || !mine || !ref || n < 0) return OTM_ERR_ARG;
    CK(exp_table_setup());
    CK(launch_exp_selftest(x, n, mine, ref, (cudaStream_t)stream));
    return OTM_OK;
}

extern "C" int otm_return_map(const otm_material *mat, double dt, int64_t n_mps, const double *dF,
                              const double *F_new, double *be, double *ebar, double *T, double *sigma, double *rate,
                              uint8_t *failed, int32_t *status, void *stream)
{
    if (!mat || !dF || !F_new || !be || !ebar || !T || !sigma || !status || n_mps < 0 || !(dt > 0))
        return OTM_ERR_ARG;
    CK(launch_return_map_only(mat, dt, n_mps, dF, F_new, be, ebar, T, sigma, rate, failed, status,
                              (cudaStream_t)stream));
    return OTM_OK;
}
