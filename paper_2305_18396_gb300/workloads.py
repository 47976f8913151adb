"""The linear products of one transformer encoder layer, as private-inference calls.

Sec. 3.1.1: every fully connected layer is one Pi_MatMul(W, <x>_0) (the client
holds <x>_0, the server W); each share-by-share attention product
(Q K^T and softmax(.) V) needs two Pi_MatMul calls for its cross terms, in the
transposed form of the footnote there so that the client always encrypts.
With seq length s, hidden width E, FFN width F and h heads of width d = E/h:

    qkv        X (s x E) . W (E x 3E)            client share . weights
    attn_out   X (s x E) . W (E x E)
    ffn1       X (s x E) . W (E x F)
    ffn2       X (s x F) . W (F x E)
    qk_x0      <Q>_0 (s x d) . <K^T>_1 (d x s)    per head: cross term 1 of Q K^T
    qk_x1      <K>_0 (s x d) . <Q>_1^T (d x s)    per head: cross term 2, transposed form
    pv_x0      <P>_0 (s x s) . <V>_1 (s x d)      per head: cross term 1 of P V
    pv_x1      <V>_0^T (d x s) . <P>_1^T (s x s)  per head: cross term 2, transposed form

(m, k, n) below is (rows of the client operand, inner dimension, columns of the
server operand).  share_weights marks products whose server operand is its
share of an activation (uniform in Z_t, encoded per request) rather than a
resident weight matrix.
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class Product:
    name: str
    m: int
    k: int
    n: int
    share_weights: bool
    count: int = 1

    @property
    def macs(self):
        return self.m * self.k * self.n * self.count


def bert_layer_products(seq=128, hidden=768, ffn=3072, heads=12, distinct_heads=None):
    """Products of one encoder layer.  With distinct_heads=1 each per-head shape appears
    once (count 1) and shapes that coincide are listed once: the distinct launches."""
    d = hidden // heads
    h = heads if distinct_heads is None else distinct_heads
    prods = [
        Product("qkv", seq, hidden, 3 * hidden, False),
        Product("attn_out", seq, hidden, hidden, False),
        Product("ffn1", seq, hidden, ffn, False),
        Product("ffn2", seq, ffn, hidden, False),
        Product("qk_x0", seq, d, seq, True, h),
        Product("qk_x1", seq, d, seq, True, h),
        Product("pv_x0", seq, seq, d, True, h),
        Product("pv_x1", d, seq, seq, True, h),
    ]
    if distinct_heads is not None:
        seen, out = set(), []
        for p in prods:
            if (p.m, p.k, p.n, p.share_weights) not in seen:
                seen.add((p.m, p.k, p.n, p.share_weights))
                out.append(p)
        prods = out
    return prods


def layer_macs(prods):
    return sum(p.macs for p in prods)


BERT_BASE = dict(seq=128, hidden=768, ffn=3072, heads=12)
BERT_LARGE = dict(seq=512, hidden=1024, ffn=4096, heads=16)
