"""GB300-native evaluation of the 3D die-to-die placement objective and its
gradient (bistratal WA wirelength + eDensity3D penalty) behind a C ABI."""
