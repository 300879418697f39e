// Runs the library's confidence kernel (csrc/confidence.cuh) under the host shim with the launch
// shape of gsparc_confidence.  Input file: int32 B, hidden; float alpha; float pos[3B],
// task_loss[B], weights[5h+1], d_weights_in[5h+1].  Output file: float objective, confidence[B],
// d_task_loss[B], d_weights[5h+1]; int32 shim violations.
#include <stdio.h>
#include <stdlib.h>

#include "cuda_emu.h"
#include "confidence.cuh"

static void rd(FILE* f, void* p, size_t n) {
    if (fread(p, 1, n, f) != n) { fprintf(stderr, "short input\n"); exit(2); }
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t B = 0, hidden = 0;
    float alpha = 0.0f;
    rd(f, &B, 4);
    rd(f, &hidden, 4);
    rd(f, &alpha, 4);
    const int nw = gsparc::conf_n_weights(hidden);
    std::vector<float> pos(3 * (size_t)B), loss(B), w(nw), dw(nw), conf(B, -1.0f), dtl(B, -1.0f);
    rd(f, pos.data(), 12 * (size_t)B);
    rd(f, loss.data(), 4 * (size_t)B);
    rd(f, w.data(), 4 * (size_t)nw);
    rd(f, dw.data(), 4 * (size_t)nw);
    fclose(f);
    float objective = -1.0f;
    emu_launch(emu_dim3{1, 1, 1}, gsparc::kConfWarps * 32, gsparc::k_confidence, (int)B, (int)hidden,
               (const float*)pos.data(), (const float*)loss.data(), (const float*)w.data(), alpha,
               (float)(1.0 / (double)B), conf.data(), &objective, dtl.data(), dw.data());
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(&objective, 4, 1, o);
    fwrite(conf.data(), 4, B, o);
    fwrite(dtl.data(), 4, B, o);
    fwrite(dw.data(), 4, nw, o);
    int32_t v = g_emu_violations.load();
    fwrite(&v, 4, 1, o);
    fclose(o);
    return 0;
}
