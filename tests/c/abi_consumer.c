/* A plain C99 consumer of include/pic.h: prints the layout of every public struct and the
 * results of the calls that need no GPU, one "key value" pair per line, for
 * tests/test_c_consumer.py to compare with the Python binding. */
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "pic.h"

#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
#define S(T) printf(#T " %zu\n", sizeof(T))

int main(void) {
    S(pic_config);
    F(pic_config, ndim); F(pic_config, nx); F(pic_config, ny); F(pic_config, nz);
    F(pic_config, dx); F(pic_config, dy); F(pic_config, dz); F(pic_config, dt);
    F(pic_config, nspecies); F(pic_config, capacity); F(pic_config, cell_capacity);
    F(pic_config, sort_interval); F(pic_config, diag_interval); F(pic_config, diag_capacity);
    F(pic_config, track_ids); F(pic_config, flags); F(pic_config, tile_x); F(pic_config, tile_y);
    F(pic_config, tile_z); F(pic_config, j_filter); F(pic_config, ctas_per_sm);
    S(pic_tune_entry); F(pic_tune_entry, tile_x); F(pic_tune_entry, tile_y); F(pic_tune_entry, ctas_per_sm);
    F(pic_tune_entry, ms_per_step);
    S(pic_species);
    F(pic_species, q); F(pic_species, m); F(pic_species, w); F(pic_species, nu);
    S(pic_diag_rec);
    F(pic_diag_rec, step); F(pic_diag_rec, t); F(pic_diag_rec, WE); F(pic_diag_rec, WB);
    F(pic_diag_rec, Ekin); F(pic_diag_rec, P); F(pic_diag_rec, flags); F(pic_diag_rec, reserved);
    S(pic_stats);
    F(pic_stats, particles); F(pic_stats, max_cell); F(pic_stats, spilled);
    F(pic_stats, cell_capacity); F(pic_stats, flags); F(pic_stats, reserved);
    S(pic_kernel_time);
    F(pic_kernel_time, name); F(pic_kernel_time, launches); F(pic_kernel_time, total_ms);
    S(pic_hybrid_config);
    F(pic_hybrid_config, nx); F(pic_hybrid_config, ny); F(pic_hybrid_config, dx);
    F(pic_hybrid_config, dy); F(pic_hybrid_config, dt); F(pic_hybrid_config, n0);
    F(pic_hybrid_config, nu); F(pic_hybrid_config, w); F(pic_hybrid_config, capacity);
    F(pic_hybrid_config, tol); F(pic_hybrid_config, max_iter); F(pic_hybrid_config, flags);
    F(pic_hybrid_config, sort_interval);
    S(pic_mlp_norm);
    F(pic_mlp_norm, mu); F(pic_mlp_norm, sigma); F(pic_mlp_norm, nin);

    pic_config c;
    memset(&c, 0, sizeof c);
    c.ndim = 2; c.nx = 64; c.ny = 64; c.nz = 1;
    c.dx = c.dy = c.dz = 0.1; c.dt = 0.05;
    c.nspecies = 2; c.capacity[0] = c.capacity[1] = 65536;
    c.sort_interval = 8; c.diag_interval = 1; c.diag_capacity = 100;
    size_t n = 0;
    printf("required_rc %d\n", pic_required_bytes(&c, &n));
    printf("required_bytes %zu\n", n);
    c.nx = 60;
    printf("bad_rc %d\n", pic_required_bytes(&c, &n));
    printf("bad_has_text %d\n", (int)(strlen(pic_last_error(NULL)) > 0));

    pic_hybrid_config h;
    memset(&h, 0, sizeof h);
    h.nx = 64; h.ny = 32; h.dx = h.dy = 0.1; h.dt = 0.05; h.n0 = 1.0; h.nu = 0.1;
    h.w = 0.1 / 16; h.capacity = 64 * 32 * 16;
    printf("hybrid_rc %d\n", pic_hybrid_required_bytes(&h, &n));
    printf("hybrid_bytes %zu\n", n);

    printf("checkpoint_null %d\n", pic_checkpoint(NULL, "x"));
    printf("loaded_null %lld\n", (long long)pic_loaded_count(NULL, 0, 0));
    printf("step_count_null %lld\n", (long long)pic_step_count(NULL));
    return 0;
}
