// warmstart.cu - the learned GS warm start: a 4-level convolutional encoder-decoder that
// maps a 256x256 target amplitude to a replay-plane phase, trained on (target, phase)
// pairs produced by gs_iterate, and used as gs_iterate's initial phase. Not part of the
// paper (its Section 3 random phase stays the fallback); an engineering extension.
//
// Network (3x3 convolutions, zero padding, stride 1; channels-last bf16 activations,
// float32 master weights, bf16 operands with float32 accumulation):
//   level 1 (256^2)  c1a 8->32, c1b 32->32 = s1          ReLU
//   level 2 (128^2)  pool(s1), c2a 32->64, c2b 64->64 = s2
//   level 3 (64^2)   pool(s2), c3a 64->128, c3b 128->128 = s3
//   level 4 (32^2)   pool(s3), c4a 128->128, c4b 128->128 = b4
//   decoder          u5 = ReLU(d5(up(b4)) + s3)  128->128 at 64^2
//                    u6 = ReLU(d6(up(u5)) + s2)  128->64  at 128^2
//                    u7 = ReLU(d7(up(u6)) + s1)  64->32   at 256^2
//   head             out = h(u7) 32->8 (channels 0, 1 = (u, v); phase = atan2(v, u))
// The input has one live channel (the target, area-averaged to 256^2) padded to 8.
// Loss: 1 - |sum_p w_p y_p conj(z_p)| / sum_p w_p with y = (u+iv)/|u+iv|, z the label
// phasor and w = target^2: invariant to a global phase offset, which GS leaves free.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "nn.h"
#include "runtime.h"

namespace holo {
namespace nn {

constexpr int kRes = 256;
constexpr int kLayers = 12;

struct LayerDesc {
    int cin, cout, div, relu;
};
// c1a c1b c2a c2b c3a c3b c4a c4b d5 d6 d7 head
static const LayerDesc kDesc[kLayers] = {
    {8, 32, 1, 1},   {32, 32, 1, 1},   {32, 64, 2, 1},   {64, 64, 2, 1},
    {64, 128, 4, 1}, {128, 128, 4, 1}, {128, 128, 8, 1}, {128, 128, 8, 1},
    {128, 128, 4, 1}, {128, 64, 2, 1},  {64, 32, 1, 1},  {32, 8, 1, 0},
};

struct Param {
    float *w, *b, *dw, *db, *mw, *vw, *mb, *vb;
    __nv_bfloat16 *wmat, *wt;
    size_t nw;
};

}  // namespace nn
}  // namespace holo

using namespace holo;
using namespace holo::nn;

struct ws_net {
    int max_batch;
    int step;
    Param p[kLayers];
    void* param_mem;
    void* act_mem;
    // activations (bf16) and their gradients
    __nv_bfloat16 *x0, *a1, *s1, *p1, *a2, *s2, *p2, *a3, *s3, *p3, *a4, *b4, *up4, *u5, *up5, *u6, *up6, *u7, *hout;
    __nv_bfloat16 *g_a1, *g_s1, *g_p1, *g_a2, *g_s2, *g_p2, *g_a3, *g_s3, *g_p3, *g_a4, *g_b4, *g_up4, *g_u5, *g_up5,
        *g_u6, *g_up6, *g_u7, *g_out;
    float* out_f32;
    float* loss_scratch;
    float* loss_dev;
    int device;
    // the batch-1 forward pass captured once as a CUDA graph (ws_infer): every buffer it
    // touches belongs to the net, so later calls only replay it
    cudaGraphExec_t infer_exec = nullptr;
    cudaGraph_t infer_graph = nullptr;
    int64_t infer_kernels = 0;   // kernels in the graph (launch accounting)
};

namespace {

size_t px(int B, int div) { return size_t(B) * (kRes / div) * (kRes / div); }

// normal variates from SplitMix64 draws (Box-Muller), deterministic in the seed
struct Rng {
    uint64_t s, k = 0;
    double uniform() {
        uint64_t z = s + (++k) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double(z >> 11) + 0.5) / 9007199254740992.0;
    }
    double normal() {
        const double u1 = uniform(), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

int conv_fwd(ws_net* n, int layer, const __nv_bfloat16* in, int B, const __nv_bfloat16* residual,
             __nv_bfloat16* out, float* out_f32, cudaStream_t st) {
    const LayerDesc& d = kDesc[layer];
    ConvArgs a{};
    a.B = B;
    a.H = a.W = kRes / d.div;
    a.Cin = d.cin;
    a.Cout = d.cout;
    a.in = in;
    a.wmat = n->p[layer].wmat;
    a.bias = n->p[layer].b;
    a.residual = residual;
    a.relu = d.relu;
    a.out = out;
    a.out_f32 = out_f32;
    return conv3x3(a, kConvFwd, st);
}

// g: gradient at the layer's output (pre-activation after relu_bwd); x: the layer input.
// Writes dx (if non-null), accumulates dW and db.
int conv_bwd(ws_net* n, int layer, const __nv_bfloat16* g, const __nv_bfloat16* x, int B, __nv_bfloat16* dx,
             cudaStream_t st) {
    const LayerDesc& d = kDesc[layer];
    int rc;
    if (dx) {
        ConvArgs a{};
        a.B = B;
        a.H = a.W = kRes / d.div;
        a.Cin = d.cout;
        a.Cout = d.cin;
        a.in = g;
        a.wmat = n->p[layer].wt;
        a.flip = 1;
        a.out = dx;
        if ((rc = conv3x3(a, kConvDgrad, st))) return rc;
    }
    ConvArgs w{};
    w.B = B;
    w.H = w.W = kRes / d.div;
    w.Cin = d.cin;
    w.Cout = d.cout;
    w.in = x;
    w.dy = g;
    w.dw = n->p[layer].dw;
    if ((rc = conv3x3(w, kConvWgrad, st))) return rc;
    return bias_grad(g, px(B, d.div), d.cout, n->p[layer].db, st);
}

int forward(ws_net* n, int B, cudaStream_t st) {
    int rc;
#define CK(x) if ((rc = (x))) return rc
    CK(conv_fwd(n, 0, n->x0, B, nullptr, n->a1, nullptr, st));
    CK(conv_fwd(n, 1, n->a1, B, nullptr, n->s1, nullptr, st));
    CK(avgpool2(n->s1, B, kRes, kRes, 32, n->p1, st));
    CK(conv_fwd(n, 2, n->p1, B, nullptr, n->a2, nullptr, st));
    CK(conv_fwd(n, 3, n->a2, B, nullptr, n->s2, nullptr, st));
    CK(avgpool2(n->s2, B, kRes / 2, kRes / 2, 64, n->p2, st));
    CK(conv_fwd(n, 4, n->p2, B, nullptr, n->a3, nullptr, st));
    CK(conv_fwd(n, 5, n->a3, B, nullptr, n->s3, nullptr, st));
    CK(avgpool2(n->s3, B, kRes / 4, kRes / 4, 128, n->p3, st));
    CK(conv_fwd(n, 6, n->p3, B, nullptr, n->a4, nullptr, st));
    CK(conv_fwd(n, 7, n->a4, B, nullptr, n->b4, nullptr, st));
    CK(upsample2(n->b4, B, kRes / 8, kRes / 8, 128, n->up4, st));
    CK(conv_fwd(n, 8, n->up4, B, n->s3, n->u5, nullptr, st));
    CK(upsample2(n->u5, B, kRes / 4, kRes / 4, 128, n->up5, st));
    CK(conv_fwd(n, 9, n->up5, B, n->s2, n->u6, nullptr, st));
    CK(upsample2(n->u6, B, kRes / 2, kRes / 2, 64, n->up6, st));
    CK(conv_fwd(n, 10, n->up6, B, n->s1, n->u7, nullptr, st));
    CK(conv_fwd(n, 11, n->u7, B, nullptr, n->hout, n->out_f32, st));
    return HOLO_OK;
}

int backward(ws_net* n, int B, cudaStream_t st) {
    int rc;
    const size_t sz1 = px(B, 1), sz2 = px(B, 2), sz4 = px(B, 4), sz8 = px(B, 8);
    for (int l = 0; l < kLayers; ++l) {
        CK(cuda_status(cudaMemsetAsync(n->p[l].dw, 0, sizeof(float) * n->p[l].nw, st), "grad reset"));
        CK(cuda_status(cudaMemsetAsync(n->p[l].db, 0, sizeof(float) * kDesc[l].cout, st), "grad reset"));
    }
    // head (linear) and decoder
    CK(conv_bwd(n, 11, n->g_out, n->u7, B, n->g_u7, st));
    CK(relu_bwd(n->g_u7, n->u7, sz1 * 32, st));
    CK(conv_bwd(n, 10, n->g_u7, n->up6, B, n->g_up6, st));
    CK(cuda_status(cudaMemcpyAsync(n->g_s1, n->g_u7, sz1 * 32 * 2, cudaMemcpyDeviceToDevice, st), "skip grad"));
    CK(upsample2_bwd(n->g_up6, B, kRes / 2, kRes / 2, 64, n->g_u6, st));
    CK(relu_bwd(n->g_u6, n->u6, sz2 * 64, st));
    CK(conv_bwd(n, 9, n->g_u6, n->up5, B, n->g_up5, st));
    CK(cuda_status(cudaMemcpyAsync(n->g_s2, n->g_u6, sz2 * 64 * 2, cudaMemcpyDeviceToDevice, st), "skip grad"));
    CK(upsample2_bwd(n->g_up5, B, kRes / 4, kRes / 4, 128, n->g_u5, st));
    CK(relu_bwd(n->g_u5, n->u5, sz4 * 128, st));
    CK(conv_bwd(n, 8, n->g_u5, n->up4, B, n->g_up4, st));
    CK(cuda_status(cudaMemcpyAsync(n->g_s3, n->g_u5, sz4 * 128 * 2, cudaMemcpyDeviceToDevice, st), "skip grad"));
    CK(upsample2_bwd(n->g_up4, B, kRes / 8, kRes / 8, 128, n->g_b4, st));
    // bottleneck and encoder
    CK(relu_bwd(n->g_b4, n->b4, sz8 * 128, st));
    CK(conv_bwd(n, 7, n->g_b4, n->a4, B, n->g_a4, st));
    CK(relu_bwd(n->g_a4, n->a4, sz8 * 128, st));
    CK(conv_bwd(n, 6, n->g_a4, n->p3, B, n->g_p3, st));
    CK(avgpool2_bwd(n->g_p3, B, kRes / 4, kRes / 4, 128, n->g_s3, 1, st));
    CK(relu_bwd(n->g_s3, n->s3, sz4 * 128, st));
    CK(conv_bwd(n, 5, n->g_s3, n->a3, B, n->g_a3, st));
    CK(relu_bwd(n->g_a3, n->a3, sz4 * 128, st));
    CK(conv_bwd(n, 4, n->g_a3, n->p2, B, n->g_p2, st));
    CK(avgpool2_bwd(n->g_p2, B, kRes / 2, kRes / 2, 64, n->g_s2, 1, st));
    CK(relu_bwd(n->g_s2, n->s2, sz2 * 64, st));
    CK(conv_bwd(n, 3, n->g_s2, n->a2, B, n->g_a2, st));
    CK(relu_bwd(n->g_a2, n->a2, sz2 * 64, st));
    CK(conv_bwd(n, 2, n->g_a2, n->p1, B, n->g_p1, st));
    CK(avgpool2_bwd(n->g_p1, B, kRes, kRes, 32, n->g_s1, 1, st));
    CK(relu_bwd(n->g_s1, n->s1, sz1 * 32, st));
    CK(conv_bwd(n, 1, n->g_s1, n->a1, B, n->g_a1, st));
    CK(relu_bwd(n->g_a1, n->a1, sz1 * 32, st));
    CK(conv_bwd(n, 0, n->g_a1, n->x0, B, nullptr, st));
    return HOLO_OK;
}

int pack_all(ws_net* n, cudaStream_t st) {
    int rc;
    for (int l = 0; l < kLayers; ++l)
        CK(pack_weights(n->p[l].w, kDesc[l].cout, kDesc[l].cin, n->p[l].wmat, n->p[l].wt, st));
    return HOLO_OK;
}
#undef CK

int check_net(const ws_net* n) {
    if (!n) return fail(HOLO_EINVAL, "ws: NULL network");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != n->device) return fail(HOLO_EINVAL, "ws: the network lives on device %d, current is %d", n->device, dev);
    return HOLO_OK;
}

}  // namespace

extern "C" int ws_net_create(ws_net** out, uint64_t seed, int max_batch) {
    clear_error();
    if (!out) return fail(HOLO_EINVAL, "ws_net_create: NULL output");
    if (max_batch < 1 || max_batch > 256) return fail(HOLO_EINVAL, "ws_net_create: max_batch %d", max_batch);
    *out = nullptr;
    ws_net* n = new ws_net();
    n->max_batch = max_batch;
    n->step = 0;
    cudaGetDevice(&n->device);
    // parameters: w b dw db mw vw mb vb (float32) + wmat wt (bf16)
    size_t fbytes = 0, hbytes = 0;
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = size_t(kDesc[l].cout) * 9 * kDesc[l].cin;
        n->p[l].nw = nw;
        fbytes += align_up(4 * nw * sizeof(float), 256) + align_up(4 * kDesc[l].cout * sizeof(float), 256);
        hbytes += 2 * align_up(nw * 2, 256);
    }
    cudaError_t e = cudaMalloc(&n->param_mem, fbytes + hbytes);
    if (e != cudaSuccess) {
        delete n;
        return fail(HOLO_ENOMEM, "ws_net_create: %s", cudaGetErrorString(e));
    }
    cudaMemset(n->param_mem, 0, fbytes + hbytes);
    char* q = static_cast<char*>(n->param_mem);
    for (int l = 0; l < kLayers; ++l) {
        const size_t nw = n->p[l].nw, nb = size_t(kDesc[l].cout);
        Param& P = n->p[l];
        P.w = reinterpret_cast<float*>(q); P.dw = P.w + nw; P.mw = P.dw + nw; P.vw = P.mw + nw;
        q += align_up(4 * nw * sizeof(float), 256);
        P.b = reinterpret_cast<float*>(q); P.db = P.b + nb; P.mb = P.db + nb; P.vb = P.mb + nb;
        q += align_up(4 * nb * sizeof(float), 256);
    }
    for (int l = 0; l < kLayers; ++l) {
        n->p[l].wmat = reinterpret_cast<__nv_bfloat16*>(q);
        q += align_up(n->p[l].nw * 2, 256);
        n->p[l].wt = reinterpret_cast<__nv_bfloat16*>(q);
        q += align_up(n->p[l].nw * 2, 256);
    }
    // He-normal weights (fan-in of the live input channels), zero biases; the head's unused
    // output channels stay zero (their gradient is zero, so Adam keeps them there)
    Rng rng{seed};
    for (int l = 0; l < kLayers; ++l) {
        const LayerDesc& d = kDesc[l];
        const int live_in = l == 0 ? 1 : d.cin;
        const int live_out = l == kLayers - 1 ? 2 : d.cout;
        const double sd = l == kLayers - 1 ? std::sqrt(1.0 / (9.0 * live_in)) : std::sqrt(2.0 / (9.0 * live_in));
        std::vector<float> w(n->p[l].nw, 0.f);
        for (int co = 0; co < live_out; ++co)
            for (int tap = 0; tap < 9; ++tap)
                for (int ci = 0; ci < live_in; ++ci) w[(size_t(co) * 9 + tap) * d.cin + ci] = float(sd * rng.normal());
        cudaMemcpy(n->p[l].w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice);
    }
    // activations and gradients for max_batch
    const int B = max_batch;
    struct Buf { __nv_bfloat16** ptr; size_t elems; };
    const size_t s1 = px(B, 1), s2 = px(B, 2), s4 = px(B, 4), s8 = px(B, 8);
    Buf bufs[] = {
        {&n->x0, s1 * 8}, {&n->a1, s1 * 32}, {&n->s1, s1 * 32}, {&n->p1, s2 * 32}, {&n->a2, s2 * 64},
        {&n->s2, s2 * 64}, {&n->p2, s4 * 64}, {&n->a3, s4 * 128}, {&n->s3, s4 * 128}, {&n->p3, s8 * 128},
        {&n->a4, s8 * 128}, {&n->b4, s8 * 128}, {&n->up4, s4 * 128}, {&n->u5, s4 * 128}, {&n->up5, s2 * 128},
        {&n->u6, s2 * 64}, {&n->up6, s1 * 64}, {&n->u7, s1 * 32}, {&n->hout, s1 * 8},
        {&n->g_a1, s1 * 32}, {&n->g_s1, s1 * 32}, {&n->g_p1, s2 * 32}, {&n->g_a2, s2 * 64}, {&n->g_s2, s2 * 64},
        {&n->g_p2, s4 * 64}, {&n->g_a3, s4 * 128}, {&n->g_s3, s4 * 128}, {&n->g_p3, s8 * 128},
        {&n->g_a4, s8 * 128}, {&n->g_b4, s8 * 128}, {&n->g_up4, s4 * 128}, {&n->g_u5, s4 * 128},
        {&n->g_up5, s2 * 128}, {&n->g_u6, s2 * 64}, {&n->g_up6, s1 * 64}, {&n->g_u7, s1 * 32},
        {&n->g_out, s1 * 8},
    };
    size_t abytes = 0;
    for (const Buf& b : bufs) abytes += align_up(b.elems * 2, 256);
    abytes += align_up(s1 * 8 * sizeof(float), 256) + align_up(sizeof(float) * (4 * B + 4), 256);
    e = cudaMalloc(&n->act_mem, abytes);
    if (e != cudaSuccess) {
        cudaFree(n->param_mem);
        delete n;
        return fail(HOLO_ENOMEM, "ws_net_create: activations (%zu bytes): %s", abytes, cudaGetErrorString(e));
    }
    q = static_cast<char*>(n->act_mem);
    for (const Buf& b : bufs) {
        *b.ptr = reinterpret_cast<__nv_bfloat16*>(q);
        q += align_up(b.elems * 2, 256);
    }
    n->out_f32 = reinterpret_cast<float*>(q);
    q += align_up(s1 * 8 * sizeof(float), 256);
    n->loss_scratch = reinterpret_cast<float*>(q);
    n->loss_dev = n->loss_scratch + 4 * B;
    int rc = pack_all(n, nullptr);
    if (rc == HOLO_OK) rc = cuda_status(cudaDeviceSynchronize(), "ws_net_create");
    if (rc) {
        cudaFree(n->act_mem);
        cudaFree(n->param_mem);
        delete n;
        return rc;
    }
    *out = n;
    return HOLO_OK;
}

extern "C" int ws_net_destroy(ws_net* net) {
    clear_error();
    if (!net) return HOLO_OK;
    if (net->infer_exec) cudaGraphExecDestroy(net->infer_exec);
    if (net->infer_graph) cudaGraphDestroy(net->infer_graph);
    cudaFree(net->act_mem);
    cudaFree(net->param_mem);
    delete net;
    return HOLO_OK;
}

extern "C" int ws_net_param_count(const ws_net* net, int64_t* count) {
    clear_error();
    if (!net || !count) return fail(HOLO_EINVAL, "ws_net_param_count: NULL argument");
    int64_t c = 0;
    for (int l = 0; l < kLayers; ++l) c += int64_t(net->p[l].nw) + kDesc[l].cout;
    *count = c;
    return HOLO_OK;
}

static int ws_grads(ws_net* net, const float* d_targets, const float* d_label, int batch, float* d_loss,
                    cudaStream_t st) {
    int rc;
    if ((rc = prep_input(d_targets, batch, kRes, kRes, kRes, kRes, net->x0, 8, st))) return rc;
    if ((rc = forward(net, batch, st))) return rc;
    if ((rc = phase_loss(net->out_f32, 8, d_label, d_targets, batch, kRes * kRes, net->loss_scratch,
                         d_loss ? d_loss : net->loss_dev, net->g_out, st)))
        return rc;
    return backward(net, batch, st);
}

extern "C" int ws_forward_backward(ws_net* net, const float* d_targets, const float* d_label_phase, int batch,
                                   float* d_loss, holo_stream_t s) {
    clear_error();
    int rc = check_net(net);
    if (rc) return rc;
    if (!d_targets || !d_label_phase || batch < 1 || batch > net->max_batch)
        return fail(HOLO_EINVAL, "ws_forward_backward: bad arguments (batch %d, max %d)", batch, net->max_batch);
    return ws_grads(net, d_targets, d_label_phase, batch, d_loss, reinterpret_cast<cudaStream_t>(s));
}

extern "C" int ws_train_step(ws_net* net, const float* d_targets, const float* d_label_phase, int batch, float lr,
                             float* d_loss, holo_stream_t s) {
    clear_error();
    int rc = check_net(net);
    if (rc) return rc;
    if (!d_targets || !d_label_phase || batch < 1 || batch > net->max_batch || !(lr > 0.f))
        return fail(HOLO_EINVAL, "ws_train_step: bad arguments (batch %d, max %d, lr %g)", batch, net->max_batch,
                    double(lr));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    if ((rc = ws_grads(net, d_targets, d_label_phase, batch, d_loss, st))) return rc;
    net->step += 1;
    for (int l = 0; l < kLayers; ++l) {
        Param& P = net->p[l];
        if ((rc = adam(P.w, P.dw, P.mw, P.vw, P.nw, lr, 0.9f, 0.999f, 1e-8f, net->step, st))) return rc;
        if ((rc = adam(P.b, P.db, P.mb, P.vb, size_t(kDesc[l].cout), lr, 0.9f, 0.999f, 1e-8f, net->step, st))) return rc;
    }
    return pack_all(net, st);
}

extern "C" int ws_infer(ws_net* net, const float* d_target, int H, int W, float* d_phase_out, holo_stream_t s) {
    clear_error();
    int rc = check_net(net);
    if (rc) return rc;
    if (!d_target || !d_phase_out || H != W || H < kRes || H % kRes)
        return fail(HOLO_EINVAL, "ws_infer: target must be square, a multiple of %d (got %dx%d)", kRes, H, W);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    if ((rc = prep_input(d_target, 1, H, W, kRes, kRes, net->x0, 8, st))) return rc;
    if (!net->infer_exec) {
        // one eager pass finishes every lazy set-up (shared-memory limits) outside the capture
        if ((rc = forward(net, 1, st))) return rc;
        if ((rc = cuda_status(cudaStreamSynchronize(st), "ws_infer: warm-up"))) return rc;
        cudaStream_t cs = nullptr;
        if ((rc = cuda_status(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "ws_infer: stream"))) return rc;
        const int prof = profiling_swap(0);   // no event timing inside a capture
        uint64_t before = 0, after = 0;
        holo_launch_count(&before);
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = forward(net, 1, cs);
            holo_launch_count(&after);
            add_launches(-int64_t(after - before));   // captured, not run
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(cs, &g);
            if (!rc && e == cudaSuccess) {
                e = cudaGraphInstantiate(&net->infer_exec, g, 0);
                if (e == cudaSuccess) net->infer_graph = g;
                else cudaGraphDestroy(g);
            } else if (g) {
                cudaGraphDestroy(g);
            }
        }
        profiling_swap(prof);
        cudaStreamDestroy(cs);
        if (rc) return rc;
        if ((rc = cuda_status(e, "ws_infer: graph capture"))) return rc;
        net->infer_kernels = int64_t(after - before);
    }
    if ((rc = cuda_status(cudaGraphLaunch(net->infer_exec, st), "ws_infer: graph launch"))) return rc;
    add_launches(net->infer_kernels);
    return phase_out(net->out_f32, 8, kRes, kRes, H, W, d_phase_out, st);
}

extern "C" int ws_phase_resample(const float* d_uv, int channels, int H, int W, int Ho, int Wo, float* d_phase,
                                 holo_stream_t s) {
    clear_error();
    if (!d_uv || !d_phase || channels < 2 || H < 1 || W < 1 || Ho < 1 || Wo < 1 ||
        int64_t(H) * W * channels > (int64_t(1) << 31) || int64_t(Ho) * Wo > (int64_t(1) << 31))
        return fail(HOLO_EINVAL, "ws_phase_resample: bad arguments (%d channels, %dx%d -> %dx%d)", channels, H, W,
                    Ho, Wo);
    return phase_out(d_uv, channels, H, W, Ho, Wo, d_phase, reinterpret_cast<cudaStream_t>(s));
}

extern "C" int ws_adam_update(float* d_w, const float* d_g, float* d_m, float* d_v, int64_t n, float lr, float beta1,
                              float beta2, float eps, int step, holo_stream_t s) {
    clear_error();
    if (!d_w || !d_g || !d_m || !d_v || n < 1 || n > (int64_t(1) << 31) || step < 1 ||
        !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
        return fail(HOLO_EINVAL, "ws_adam_update: bad arguments (n %lld, step %d)", (long long)n, step);
    return adam(d_w, d_g, d_m, d_v, size_t(n), lr, beta1, beta2, eps, step, reinterpret_cast<cudaStream_t>(s));
}

// which: 0 weights [Cout][3][3][Cin], 1 biases [Cout], 2 weight gradients, 3 bias gradients
extern "C" int ws_get_tensor(const ws_net* net, int layer, int which, float* h_out, int64_t count) {
    clear_error();
    if (!net || !h_out || layer < 0 || layer >= kLayers || which < 0 || which > 3)
        return fail(HOLO_EINVAL, "ws_get_tensor: bad arguments");
    const Param& P = net->p[layer];
    const size_t n = (which == 0 || which == 2) ? P.nw : size_t(kDesc[layer].cout);
    if (count != int64_t(n)) return fail(HOLO_EINVAL, "ws_get_tensor: count %lld, tensor has %zu", (long long)count, n);
    const float* src = which == 0 ? P.w : which == 1 ? P.b : which == 2 ? P.dw : P.db;
    return cuda_status(cudaMemcpy(h_out, src, sizeof(float) * n, cudaMemcpyDeviceToHost), "ws_get_tensor");
}

extern "C" int ws_set_tensor(ws_net* net, int layer, int which, const float* h_in, int64_t count) {
    clear_error();
    if (!net || !h_in || layer < 0 || layer >= kLayers || which < 0 || which > 1)
        return fail(HOLO_EINVAL, "ws_set_tensor: bad arguments");
    Param& P = net->p[layer];
    const size_t n = which == 0 ? P.nw : size_t(kDesc[layer].cout);
    if (count != int64_t(n)) return fail(HOLO_EINVAL, "ws_set_tensor: count %lld, tensor has %zu", (long long)count, n);
    int rc = cuda_status(cudaMemcpy(which == 0 ? P.w : P.b, h_in, sizeof(float) * n, cudaMemcpyHostToDevice),
                         "ws_set_tensor");
    if (rc) return rc;
    return pack_all(net, nullptr);
}

extern "C" int ws_layer_shape(int layer, int* cin, int* cout, int* resolution) {
    clear_error();
    if (layer < 0 || layer >= kLayers || !cin || !cout || !resolution) return fail(HOLO_EINVAL, "ws_layer_shape");
    *cin = kDesc[layer].cin;
    *cout = kDesc[layer].cout;
    *resolution = kRes / kDesc[layer].div;
    return HOLO_OK;
}

// host float32 copy of a stored activation or activation gradient of sample 0..batch-1
extern "C" int ws_get_activation(const ws_net* net, const char* name, int batch, float* h_out, int64_t count) {
    clear_error();
    if (!net || !name || !h_out || batch < 1 || batch > net->max_batch)
        return fail(HOLO_EINVAL, "ws_get_activation: bad arguments");
    struct Entry { const char* name; const __nv_bfloat16* p; int c, div; };
    const Entry tab[] = {
        {"x0", net->x0, 8, 1}, {"a1", net->a1, 32, 1}, {"s1", net->s1, 32, 1}, {"p1", net->p1, 32, 2},
        {"a2", net->a2, 64, 2}, {"s2", net->s2, 64, 2}, {"p2", net->p2, 64, 4}, {"a3", net->a3, 128, 4},
        {"s3", net->s3, 128, 4}, {"p3", net->p3, 128, 8}, {"a4", net->a4, 128, 8}, {"b4", net->b4, 128, 8},
        {"up4", net->up4, 128, 4}, {"u5", net->u5, 128, 4}, {"up5", net->up5, 128, 2}, {"u6", net->u6, 64, 2},
        {"up6", net->up6, 64, 1}, {"u7", net->u7, 32, 1}, {"g_out", net->g_out, 8, 1}, {"g_u7", net->g_u7, 32, 1},
        {"g_up6", net->g_up6, 64, 1}, {"g_u6", net->g_u6, 64, 2}, {"g_s1", net->g_s1, 32, 1},
    };
    if (strcmp(name, "out") == 0) {
        const size_t n = px(batch, 1) * 8;
        if (count != int64_t(n)) return fail(HOLO_EINVAL, "ws_get_activation: count %lld != %zu", (long long)count, n);
        return cuda_status(cudaMemcpy(h_out, net->out_f32, sizeof(float) * n, cudaMemcpyDeviceToHost), "ws_get_activation");
    }
    for (const Entry& e : tab) {
        if (strcmp(name, e.name) != 0) continue;
        const size_t n = px(batch, e.div) * e.c;
        if (count != int64_t(n)) return fail(HOLO_EINVAL, "ws_get_activation: count %lld != %zu", (long long)count, n);
        std::vector<__nv_bfloat16> tmp(n);
        int rc = cuda_status(cudaMemcpy(tmp.data(), e.p, 2 * n, cudaMemcpyDeviceToHost), "ws_get_activation");
        if (rc) return rc;
        for (size_t i = 0; i < n; ++i) h_out[i] = __bfloat162float(tmp[i]);
        return HOLO_OK;
    }
    return fail(HOLO_EINVAL, "ws_get_activation: unknown tensor %s", name);
}

extern "C" int ws_save(const ws_net* net, const char* path) {
    clear_error();
    if (!net || !path) return fail(HOLO_EINVAL, "ws_save: NULL argument");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(HOLO_EINVAL, "ws_save: cannot open %s", path);
    const char magic[8] = {'H', 'O', 'L', 'O', 'W', 'S', '0', '1'};
    fwrite(magic, 1, 8, f);
    fwrite(&net->step, sizeof(int), 1, f);
    std::vector<float> buf;
    for (int l = 0; l < kLayers; ++l) {
        const Param& P = net->p[l];
        const size_t nb = size_t(kDesc[l].cout);
        const float* srcs[6] = {P.w, P.b, P.mw, P.vw, P.mb, P.vb};
        const size_t cnt[6] = {P.nw, nb, P.nw, P.nw, nb, nb};
        for (int k = 0; k < 6; ++k) {
            buf.resize(cnt[k]);
            cudaMemcpy(buf.data(), srcs[k], sizeof(float) * cnt[k], cudaMemcpyDeviceToHost);
            fwrite(buf.data(), sizeof(float), cnt[k], f);
        }
    }
    fclose(f);
    return cuda_status(cudaGetLastError(), "ws_save");
}

extern "C" int ws_load(ws_net* net, const char* path) {
    clear_error();
    if (!net || !path) return fail(HOLO_EINVAL, "ws_load: NULL argument");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(HOLO_EINVAL, "ws_load: cannot open %s", path);
    char magic[8];
    int step = 0;
    if (fread(magic, 1, 8, f) != 8 || memcmp(magic, "HOLOWS01", 8) != 0 || fread(&step, sizeof(int), 1, f) != 1) {
        fclose(f);
        return fail(HOLO_EINVAL, "ws_load: %s is not a warm-start checkpoint", path);
    }
    std::vector<float> buf;
    for (int l = 0; l < kLayers; ++l) {
        Param& P = net->p[l];
        const size_t nb = size_t(kDesc[l].cout);
        float* dsts[6] = {P.w, P.b, P.mw, P.vw, P.mb, P.vb};
        const size_t cnt[6] = {P.nw, nb, P.nw, P.nw, nb, nb};
        for (int k = 0; k < 6; ++k) {
            buf.resize(cnt[k]);
            if (fread(buf.data(), sizeof(float), cnt[k], f) != cnt[k]) {
                fclose(f);
                return fail(HOLO_EINVAL, "ws_load: %s is truncated", path);
            }
            cudaMemcpy(dsts[k], buf.data(), sizeof(float) * cnt[k], cudaMemcpyHostToDevice);
        }
    }
    fclose(f);
    net->step = step;
    return pack_all(net, nullptr);
}

// ------------------------------------------------------------ primitives ----
extern "C" int nn_conv3x3(int mode, int B, int H, int W, int Cin, int Cout, const void* d_in, const void* d_wmat,
                          const void* d_dy, const float* d_bias, const void* d_residual, int relu, void* d_out,
                          float* d_out_f32, float* d_dw, holo_stream_t s) {
    clear_error();
    const bool legacy = (mode & HOLO_CONV_LEGACY) != 0;
    mode &= ~HOLO_CONV_LEGACY;
    if (mode < 0 || mode > 2 || B < 1 || H < 1 || W < 1 || Cin < 8 || Cout < 8 || Cin % 8 || Cout % 8 || !d_in)
        return fail(HOLO_EINVAL, "nn_conv3x3: bad arguments");
    ConvArgs a{};
    a.B = B;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.in = static_cast<const __nv_bfloat16*>(d_in);
    a.wmat = static_cast<const __nv_bfloat16*>(d_wmat);
    a.dy = static_cast<const __nv_bfloat16*>(d_dy);
    a.bias = d_bias;
    a.residual = static_cast<const __nv_bfloat16*>(d_residual);
    a.relu = relu;
    a.flip = mode == kConvDgrad;
    a.out = static_cast<__nv_bfloat16*>(d_out);
    a.out_f32 = d_out_f32;
    a.dw = d_dw;
    if (mode != kConvWgrad && (!d_wmat || (!d_out && !d_out_f32))) return fail(HOLO_EINVAL, "nn_conv3x3: outputs");
    if (mode == kConvWgrad && (!d_dy || !d_dw)) return fail(HOLO_EINVAL, "nn_conv3x3: wgrad needs dy and dw");
    return conv3x3(a, mode, reinterpret_cast<cudaStream_t>(s), legacy);
}

extern "C" int holo_tc_status(int* fault, int clear) {
    clear_error();
    if (!fault) return fail(HOLO_EINVAL, "holo_tc_status: NULL output");
    int a = 0, b = 0, c = 0, d = 0;
    int rc = conv3x3_tc05_fault(&a, clear != 0);
    if (rc) return rc;
    if ((rc = holo::ospr_tc05_fault(&b, clear != 0))) return rc;
    if ((rc = holo::ospr_persistent_fault(&c, clear != 0))) return rc;
    if ((rc = holo::gs_tc05_fault(&d, clear != 0))) return rc;
    *fault = a | b | c | d;
    return HOLO_OK;
}
