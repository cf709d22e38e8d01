/*
 * oracle/cnn.c -- plain FP64 reference for the learned warm-start refiner.
 *
 * TEST INFRASTRUCTURE ONLY (see radon.c).
 *
 * The paper has no learned component; this refiner of the filtered back-projection
 * start is an addition: four 3x3 convolutions with 32 channels.  Reading used here: channels 1 -> 32 -> 32 -> 32 -> 1, zero padding
 * of one pixel, a bias per output channel, ReLU after the first three layers, none
 * after the last.  The network maps a normalised FBP image to a correction (the caller
 * forms x' = x + s * net(x / s)).
 *
 * Parameter layout (doubles), layer l = 0..3 with (cin, cout) = (1,32), (32,32), (32,32),
 * (32,1): weights W_l[cout][cin][3][3] followed by bias b_l[cout]; layers back to back.
 * Total 19105 values.
 */
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

static const int CIN[4] = {1, 32, 32, 32};
static const int COUT[4] = {32, 32, 32, 1};

int orc_cnn_param_count(void)
{
    int n = 0;
    for (int l = 0; l < 4; ++l) n += COUT[l] * CIN[l] * 9 + COUT[l];
    return n;
}

static const double *layer_w(const double *p, int l)
{
    for (int i = 0; i < l; ++i) p += COUT[i] * CIN[i] * 9 + COUT[i];
    return p;
}

/* out[co][y][x] = b[co] + sum_ci sum_{dy,dx} W[co][ci][dy+1][dx+1] in[ci][y+dy][x+dx] */
static void conv3x3(const double *in, int cin, int H, int Wd, const double *w, int cout, double *out)
{
    const double *bias = w + (size_t)cout * cin * 9;
    for (int co = 0; co < cout; ++co) {
        for (int y = 0; y < H; ++y) {
            for (int x = 0; x < Wd; ++x) {
                double acc = bias[co];
                for (int ci = 0; ci < cin; ++ci) {
                    for (int dy = -1; dy <= 1; ++dy) {
                        int yy = y + dy;
                        if (yy < 0 || yy >= H) continue;
                        for (int dx = -1; dx <= 1; ++dx) {
                            int xx = x + dx;
                            if (xx < 0 || xx >= Wd) continue;
                            acc += w[((size_t)(co * cin + ci) * 3 + (dy + 1)) * 3 + (dx + 1)] *
                                   in[((size_t)ci * H + yy) * Wd + xx];
                        }
                    }
                }
                out[((size_t)co * H + y) * Wd + x] = acc;
            }
        }
    }
}

/* Forward for a batch of B single-channel H x W images; act (may be NULL) receives the
 * post-ReLU activations of layers 0..2, [B][3][32][H][W]. */
void orc_cnn_forward(const double *in, int B, int H, int Wd, const double *params, double *out)
{
    size_t plane = (size_t)H * Wd;
    double *a = malloc(sizeof(double) * 32 * plane);
    double *b = malloc(sizeof(double) * 32 * plane);
    for (int n = 0; n < B; ++n) {
        const double *src = in + n * plane;
        conv3x3(src, 1, H, Wd, layer_w(params, 0), 32, a);
        for (size_t i = 0; i < 32 * plane; ++i) a[i] = a[i] > 0 ? a[i] : 0;
        conv3x3(a, 32, H, Wd, layer_w(params, 1), 32, b);
        for (size_t i = 0; i < 32 * plane; ++i) b[i] = b[i] > 0 ? b[i] : 0;
        conv3x3(b, 32, H, Wd, layer_w(params, 2), 32, a);
        for (size_t i = 0; i < 32 * plane; ++i) a[i] = a[i] > 0 ? a[i] : 0;
        conv3x3(a, 32, H, Wd, layer_w(params, 3), 1, out + n * plane);
    }
    free(a);
    free(b);
}

/* Backward of L = sum(gout * net(in)): gparams (accumulated into, same layout as params)
 * and gin (overwritten, may be NULL). */
void orc_cnn_backward(const double *in, int B, int H, int Wd, const double *params, const double *gout,
                      double *gparams, double *gin)
{
    size_t plane = (size_t)H * Wd;
    double *act[4];
    for (int l = 0; l < 4; ++l) act[l] = malloc(sizeof(double) * 32 * plane);
    double *gcur = malloc(sizeof(double) * 32 * plane);
    double *gprev = malloc(sizeof(double) * 32 * plane);
    for (int n = 0; n < B; ++n) {
        /* forward, keeping the layer inputs: act[0] = input, act[1..3] = post-ReLU outputs */
        memcpy(act[0], in + n * plane, sizeof(double) * plane);
        for (int l = 0; l < 3; ++l) {
            conv3x3(act[l], CIN[l], H, Wd, layer_w(params, l), COUT[l], act[l + 1]);
            for (size_t i = 0; i < (size_t)COUT[l] * plane; ++i) act[l + 1][i] = act[l + 1][i] > 0 ? act[l + 1][i] : 0;
        }
        memcpy(gcur, gout + n * plane, sizeof(double) * plane);
        for (int l = 3; l >= 0; --l) {
            int cin = CIN[l], cout = COUT[l];
            const double *w = layer_w(params, l);
            double *gw = (double *)layer_w(gparams, l);
            double *gb = gw + (size_t)cout * cin * 9;
            /* gcur is dL/d(pre-activation output of layer l) */
            for (int co = 0; co < cout; ++co)
                for (size_t i = 0; i < plane; ++i) gb[co] += gcur[co * plane + i];
            for (int co = 0; co < cout; ++co)
                for (int ci = 0; ci < cin; ++ci)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            double acc = 0.0;
                            for (int y = 0; y < H; ++y) {
                                int yy = y + dy;
                                if (yy < 0 || yy >= H) continue;
                                for (int x = 0; x < Wd; ++x) {
                                    int xx = x + dx;
                                    if (xx < 0 || xx >= Wd) continue;
                                    acc += gcur[((size_t)co * H + y) * Wd + x] * act[l][((size_t)ci * H + yy) * Wd + xx];
                                }
                            }
                            gw[((size_t)(co * cin + ci) * 3 + (dy + 1)) * 3 + (dx + 1)] += acc;
                        }
            /* dL/d(input of layer l) */
            for (int ci = 0; ci < cin; ++ci)
                for (int y = 0; y < H; ++y)
                    for (int x = 0; x < Wd; ++x) {
                        double acc = 0.0;
                        for (int co = 0; co < cout; ++co)
                            for (int dy = -1; dy <= 1; ++dy) {
                                int yo = y - dy;
                                if (yo < 0 || yo >= H) continue;
                                for (int dx = -1; dx <= 1; ++dx) {
                                    int xo = x - dx;
                                    if (xo < 0 || xo >= Wd) continue;
                                    acc += w[((size_t)(co * cin + ci) * 3 + (dy + 1)) * 3 + (dx + 1)] *
                                           gcur[((size_t)co * H + yo) * Wd + xo];
                                }
                            }
                        gprev[((size_t)ci * H + y) * Wd + x] = acc;
                    }
            if (l > 0) {
                /* through the ReLU that produced act[l] */
                for (size_t i = 0; i < (size_t)cin * plane; ++i) gcur[i] = act[l][i] > 0 ? gprev[i] : 0.0;
            } else if (gin) {
                memcpy(gin + n * plane, gprev, sizeof(double) * plane);
            }
        }
    }
    for (int l = 0; l < 4; ++l) free(act[l]);
    free(gcur);
    free(gprev);
}
