"""FP64 CPU oracle for Compressive Spectral Clustering (Tremblay et al., ICML 2016).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: it exists so that the tests, ``__graft_entry__.smoke()``
and the benchmark's ``cpu_baseline`` / reference leg can check and time the
CUDA path against a plain, slow, obviously correct restatement of the paper.
It shares no code, tables or constants generation with the CUDA library;
the only inputs the two sides have in common come from ``csc_inputs``.

Modules, each following the passage it cites:

* ``laplacian``  normalized Laplacian L = I - D^-1/2 W D^-1/2 (Sec. 2.1).
* ``chebyshev``  Jackson-Chebyshev approximation of the ideal low-pass filter
  (Eq. 1, Sec. 2.1 "Fast graph filtering", Sec. 4.3), the filtered block of
  Alg. 2 step 4, eigencount moments and the dichotomy of Sec. 4.3.
* ``rng``        Philox4x32-10 and SplitMix64, written from their published
  definitions, with the Box-Muller transform (Alg. 2 step 3).
* ``sampling``   uniform sampling without replacement (Sec. 3.2, Eq. 4).
* ``kmeans``     k-means++ seeding and Lloyd iterations (Alg. 2 step 6).
* ``interp``     the interpolation problem of Eq. 5 and the label rule of Sec. 4.1.
* ``ari``        adjusted Rand index (Hubert & Arabie 1985, Sec. 5.2).
* ``pipeline``   Alg. 2 end to end.
* ``mlp``        FP64 forward/backward of the bracket-predicting MLP.
* ``bracket``    features and targets of the learned lambda_k bracket (the eigencount
  of Sec. 4.3 still decides whether the predicted interval holds an answer).
* ``sc``         dense spectral clustering, Alg. 1 (Sec. 2.2), the comparison baseline
  of the small recovery sweeps.

Parity status of every function is stated in its module header; functions
without an independent pin say "parity unpinned".
"""
