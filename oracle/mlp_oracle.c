/*
 * mlp_oracle.c -- ORACLE for the learned Trotter-column proposal (not in the
 * paper; an addition built on its QMC setting of M identical slices, section
 * 3.1).  TEST INFRASTRUCTURE ONLY, plain FP64, no code shared with the CUDA
 * library.
 *
 * Column x (site q of a model with M slices) of one replica at inverse
 * temperature beta.  phi_t = h_q + sum_{q' spatial nbr} J_qq' s_{q',t} is the
 * spatial field of spin (q,t); it does not depend on the column's own spins.
 * The column's share of the cost function (section 1) is
 *     E_col(s) = -sum_t s_t phi_t - Jtau sum_{t} s_t s_{t+1 mod M}
 * (for M = 2 the single Trotter edge, for M = 1 no Trotter term), so the
 * conditional law of the column given everything else is exp(-beta E_col).
 *
 * Network: input x = (phi_0/8 .. phi_{M-1}/8, beta), ReLU hidden layers
 *     h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), l = W3 h2 + b3,
 * l_t the logit of P(s'_t = +1).  Loss per sample: sum_t softplus(l_t) - y_t l_t
 * (Bernoulli negative log-likelihood, y_t = (s_t + 1)/2), averaged over the
 * batch.  The proposal q(s') = prod_t sigma(s'_t l_t) is independent of the
 * current column, so the Metropolis-Hastings log ratio of s -> s' is
 *     log A = -beta (E_col(s') - E_col(s)) + log q(s) - log q(s').
 *
 * Flip-symmetric mixture: q_mix(s') = (q(s') + q(-s')) / 2, drawn by taking
 * q's draw or its complement with probability 1/2 each.  It is again
 * independent of the current column, so the same ratio holds with q_mix in
 * place of q.  (A column aligned along the Trotter ring then has its whole
 * reversal as a likely proposal.)
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Forward pass for B samples.  X [B][IN], W1 [H][IN], W2 [H][H], W3 [OUT][H]. */
void orc_mlp_forward(int B, int IN, int H, int OUT, const double* X, const double* W1,
                     const double* b1, const double* W2, const double* b2, const double* W3,
                     const double* b3, double* H1, double* H2, double* L)
{
    for (int b = 0; b < B; b++) {
        const double* x = X + (int64_t)b * IN;
        double* h1 = H1 + (int64_t)b * H;
        double* h2 = H2 + (int64_t)b * H;
        double* l = L + (int64_t)b * OUT;
        for (int j = 0; j < H; j++) {
            double a = b1[j];
            for (int i = 0; i < IN; i++)
                a += W1[(int64_t)j * IN + i] * x[i];
            h1[j] = a > 0 ? a : 0;
        }
        for (int j = 0; j < H; j++) {
            double a = b2[j];
            for (int i = 0; i < H; i++)
                a += W2[(int64_t)j * H + i] * h1[i];
            h2[j] = a > 0 ? a : 0;
        }
        for (int j = 0; j < OUT; j++) {
            double a = b3[j];
            for (int i = 0; i < H; i++)
                a += W3[(int64_t)j * H + i] * h2[i];
            l[j] = a;
        }
    }
}

/* Mean Bernoulli NLL over the batch and its gradient with respect to every
 * weight and bias (plain backpropagation through the three layers).  Y [B][OUT]
 * holds 0/1 targets.  Returns the loss. */
double orc_mlp_backward(int B, int IN, int H, int OUT, const double* X, const double* Y,
                        const double* W1, const double* b1, const double* W2, const double* b2,
                        const double* W3, const double* b3, double* dW1, double* db1,
                        double* dW2, double* db2, double* dW3, double* db3, double* scratch)
{
    /* scratch: H1, H2, L [B][*] followed by per-sample dL, dH2, dH1 */
    double* H1 = scratch;
    double* H2 = H1 + (int64_t)B * H;
    double* L = H2 + (int64_t)B * H;
    double* dl = L + (int64_t)B * OUT;
    double* dh2 = dl + OUT;
    double* dh1 = dh2 + H;
    orc_mlp_forward(B, IN, H, OUT, X, W1, b1, W2, b2, W3, b3, H1, H2, L);
    memset(dW1, 0, sizeof(double) * H * IN);
    memset(db1, 0, sizeof(double) * H);
    memset(dW2, 0, sizeof(double) * H * H);
    memset(db2, 0, sizeof(double) * H);
    memset(dW3, 0, sizeof(double) * OUT * H);
    memset(db3, 0, sizeof(double) * OUT);
    double loss = 0;
    for (int b = 0; b < B; b++) {
        const double* x = X + (int64_t)b * IN;
        const double* y = Y + (int64_t)b * OUT;
        const double* h1 = H1 + (int64_t)b * H;
        const double* h2 = H2 + (int64_t)b * H;
        const double* l = L + (int64_t)b * OUT;
        for (int j = 0; j < OUT; j++) {
            loss += softplus(l[j]) - y[j] * l[j];
            dl[j] = (sigmoid(l[j]) - y[j]) / B;
            db3[j] += dl[j];
            for (int i = 0; i < H; i++)
                dW3[(int64_t)j * H + i] += dl[j] * h2[i];
        }
        for (int i = 0; i < H; i++) {
            double a = 0;
            for (int j = 0; j < OUT; j++)
                a += dl[j] * W3[(int64_t)j * H + i];
            dh2[i] = h2[i] > 0 ? a : 0;
            db2[i] += dh2[i];
            for (int k = 0; k < H; k++)
                dW2[(int64_t)i * H + k] += dh2[i] * h1[k];
        }
        for (int i = 0; i < H; i++) {
            double a = 0;
            for (int j = 0; j < H; j++)
                a += dh2[j] * W2[(int64_t)j * H + i];
            dh1[i] = h1[i] > 0 ? a : 0;
            db1[i] += dh1[i];
            for (int k = 0; k < IN; k++)
                dW1[(int64_t)i * IN + k] += dh1[i] * x[k];
        }
    }
    return loss / B;
}

/* Column energy E_col(s) for M slices (see the file header). */
int64_t orc_column_energy(int M, int jtau, const int32_t* phi, const int8_t* s)
{
    int64_t e = 0;
    for (int t = 0; t < M; t++)
        e -= (int64_t)s[t] * phi[t];
    if (M >= 3) {
        for (int t = 0; t < M; t++)
            e -= (int64_t)jtau * s[t] * s[(t + 1) % M];
    } else if (M == 2) {
        e -= (int64_t)jtau * s[0] * s[1];
    }
    return e;
}

/* log q(s) = sum_t log sigma(s_t l_t) for the independent-Bernoulli proposal. */
double orc_log_q(int M, const double* logits, const int8_t* s)
{
    double a = 0;
    for (int t = 0; t < M; t++)
        a -= softplus(-(double)s[t] * logits[t]);
    return a;
}

/* log q_mix(s) = log((q(s) + q(-s)) / 2), formed as the log of a sum of two
 * exponentials. */
double orc_log_q_mix(int M, const double* logits, const int8_t* s)
{
    int8_t neg[64];
    for (int t = 0; t < M; t++)
        neg[t] = (int8_t)-s[t];
    const double a = orc_log_q(M, logits, s), b = orc_log_q(M, logits, neg);
    const double m = a > b ? a : b;
    return m + log(0.5 * exp(a - m) + 0.5 * exp(b - m));
}

/* MH log ratio of the move s -> s2 under the mixture proposal; dE as below. */
double orc_column_log_accept_mix(int M, int jtau, const int32_t* phi, const int8_t* s,
                                 const int8_t* s2, const double* logits, double beta, int64_t* dE)
{
    const int64_t d = orc_column_energy(M, jtau, phi, s2) - orc_column_energy(M, jtau, phi, s);
    if (dE)
        *dE = d;
    return -beta * (double)d + orc_log_q_mix(M, logits, s) - orc_log_q_mix(M, logits, s2);
}

/* MH log ratio of the move s -> s2 (see the file header); dE receives
 * E_col(s2) - E_col(s). */
double orc_column_log_accept(int M, int jtau, const int32_t* phi, const int8_t* s,
                             const int8_t* s2, const double* logits, double beta, int64_t* dE)
{
    const int64_t d = orc_column_energy(M, jtau, phi, s2) - orc_column_energy(M, jtau, phi, s);
    if (dE)
        *dE = d;
    return -beta * (double)d + orc_log_q(M, logits, s) - orc_log_q(M, logits, s2);
}
